// Stripe gather: the consumer of the H -> H' map for fp16 tiles whose run
// stride Ks*Kt is 1 mod 4 (every odd square cut-out, among others).  It
// replaces eight 2-byte shared loads per 16-byte output chunk by 16-byte
// loads and a lane exchange; for fp32 (four loads per chunk) it measured
// slower than the chunk path of lfbp_device.cuh, which fp32 tiles keep.
//
// Inside one tile row j the map reads output element (q, v) of run q from
// segment b = (q + v - c_t) mod Ny at pixel t = Kt-1-v: a walk along a
// diagonal of the stage (b+1, t-1).  Element (q+k, v+g-k) for k = 0..3 sits
// in segment B+g at consecutive pixels, i.e. four consecutive stage elements
// of one segment hold one element of each of four neighbouring runs, on an
// anti-diagonal of the (q, v) plane.  So four lanes g = 0..3 that read such
// 4-element windows from segments B..B+3 hold, together, a 4 x 4 block whose
// transpose is four output chunks: after a 4 x 4 exchange across the lanes
// (shuffles), lane k holds 4 consecutive elements (16 bytes in fp32, 8 in
// fp16) of run q+k starting at column v-k.  Because Ks*Kt = 1 (mod 4), the
// runs q..q+3 have the same alignment shift, so one choice of v aligns all
// four chunks.
//
// STRIPE.  The windows of run blocks q, q+4, q+8, ... at columns v, v-4,
// v-8, ... come from the same four segments, one window after the other: a
// lane reads one contiguous stretch of its segment (S windows) with aligned
// 16-byte shared loads and cuts the S windows out in registers (their common
// misalignment is the segment's phase, a run-time value).  A stripe is (row
// j, band of S run blocks, start column); a warp takes eight stripes per
// step.  Chunks that straddle two rows of the tile (or a run's ends) are left
// to an edge pass that moves them element by element.
#pragma once

namespace lfbp {

// Byte permute of the pair (a, b): result byte i is byte sel[4i+2:4i] of the
// eight bytes a0..a3 b0..b3 (selector values 0..7 only).
__host__ __device__ __forceinline__ uint32_t perm_bytes(uint32_t a, uint32_t b, uint32_t sel) {
#ifdef __CUDA_ARCH__
  return __byte_perm(a, b, sel);
#else
  const uint64_t x = ((uint64_t)b << 32) | a;
  uint32_t r = 0;
  for (int i = 0; i < 4; ++i) r |= (uint32_t)((x >> (8 * ((sel >> (4 * i)) & 7))) & 0xffu) << (8 * i);
  return r;
#endif
}

// ---------------------------------------------------------------- exchange --
// The 4 x 4 transpose across the lanes g = 0..3 of a group, as two exchange
// stages (partner g^2, then g^1).  Each stage is: every lane computes what it
// sends (xs_*), receives its partner's value, and updates its registers
// (xr_*).  The functions are per lane and pure, so the host emulation runs
// the same code with the exchange done through arrays.
//
// fp32: lane g holds r[k] = M[g][k]; afterwards r[k] = M[k][g].
__host__ __device__ inline void xs_a32(const uint32_t r[4], int g, uint32_t s[2]) {
  const bool hi = g & 2;
  s[0] = hi ? r[0] : r[2];
  s[1] = hi ? r[1] : r[3];
}
__host__ __device__ inline void xr_a32(uint32_t r[4], int g, const uint32_t x[2]) {
  const bool hi = g & 2;
  r[0] = hi ? x[0] : r[0];
  r[1] = hi ? x[1] : r[1];
  r[2] = hi ? r[2] : x[0];
  r[3] = hi ? r[3] : x[1];
}
__host__ __device__ inline void xs_b32(const uint32_t r[4], int g, uint32_t s[2]) {
  const bool odd = g & 1;
  s[0] = odd ? r[0] : r[1];
  s[1] = odd ? r[2] : r[3];
}
__host__ __device__ inline void xr_b32(uint32_t r[4], int g, const uint32_t x[2]) {
  const bool odd = g & 1;
  r[0] = odd ? x[0] : r[0];
  r[1] = odd ? r[1] : x[0];
  r[2] = odd ? x[1] : r[2];
  r[3] = odd ? r[3] : x[1];
}
// fp16: lane g holds w[0] = (M[g][0], M[g][1]), w[1] = (M[g][2], M[g][3])
// (low half first); afterwards w[0] = (M[0][g], M[1][g]), w[1] = (M[2][g], M[3][g]).
__host__ __device__ inline uint32_t xs_a16(const uint32_t w[2], int g) { return (g & 2) ? w[0] : w[1]; }
__host__ __device__ inline void xr_a16(uint32_t w[2], int g, uint32_t x) {
  const bool hi = g & 2;
  w[0] = hi ? x : w[0];
  w[1] = hi ? w[1] : x;
}
__host__ __device__ inline uint32_t xs_b16(const uint32_t w[2], int g) {
  // even lanes send the high halves of both words, odd lanes the low halves
  return perm_bytes(w[0], w[1], (g & 1) ? 0x5410 : 0x7632);
}
__host__ __device__ inline void xr_b16(uint32_t w[2], int g, uint32_t x) {
  // odd lanes: x = partner's (w0.hi, w1.hi): new w0 = (x.lo, w0.hi), w1 = (x.hi, w1.hi);
  // even lanes: x = partner's (w0.lo, w1.lo): new w0 = (w0.lo, x.lo), w1 = (w1.lo, x.hi)
  const bool odd = g & 1;
  w[0] = perm_bytes(w[0], x, odd ? 0x3254u : 0x5410u);
  w[1] = perm_bytes(w[1], x, odd ? 0x3276u : 0x7610u);
}

// Lane g's stream over the stretch of its segment that holds the S windows
// of one stripe: the stretch starts at the 16-byte boundary A (stage
// element) at or below the first window, whose misalignment is d; window i
// (slots k = 0..3 for runs q0 + 4i + k) starts d + 4i elements after A.  Only
// the two 16-byte vectors that window i touches are held: the window of
// fp32 i lies in vectors i, i+1; the fp16 windows 2m and 2m+1 lie in vectors
// m, m+1.
struct StripeStream {
  int A, d;
  uint4 va, vb;
};

// Position of stripe `item` of the tile (item < c.nitems_s): row j, first run
// block rb0 and start column V (the column of run block rb0's chunks).
struct StripePos {
  int j, q0, V, B, rb;  // rb: the row's row-base entry
};

template <int S>
__device__ __forceinline__ StripePos stripe_pos(const TileCtx& c, int item) {
  StripePos s;
  const int band = (int)fdiv((uint32_t)item, c.frowns);
  const int rem = item - band * c.rowns;
  s.j = (int)fdiv((uint32_t)rem, c.fns);
  const int n = rem - s.j * c.ns;
  const int alpha = (-(c.om0 + s.j * c.ncols)) & 3;  // aligns run block 0 (and every block)
  s.V = alpha + 4 * n;
  s.q0 = 4 * S * band;
  s.B = (int)fmod_((uint32_t)(s.q0 + c.cb + s.V), c.fNy);
  s.rb = tab_load(c, s.j);
  return s;
}

// 16-byte vector v of the stretch, clamped into the tile's stage (windows of
// chunks outside the row read elements that are never stored).
template <int ES>
__device__ __forceinline__ uint4 stripe_vec(const TileCtx& c, const StripeStream& st, int v) {
  int off = (st.A + v * (16 / ES)) * ES;
  const int hi = c.tile_bytes - 16;
  off = off < 0 ? 0 : (off > hi ? hi : off);
  return lds_v4(c, c.stage_s + (uint32_t)off);
}

// Start of lane g's stream for one stripe: the stretch's position and the
// first vector(s).
template <int ES>
__device__ __forceinline__ void stripe_begin(const TileCtx& c, const StripePos& sp, int g,
                                             StripeStream& st) {
  constexpr int E = 16 / ES;
  int b = sp.B + g;
  if (b >= c.Ny) b -= c.Ny;
  const int X = sp.rb + b * c.P - sp.V - g;  // stage element of slot 0 of window 0
  st.A = X & ~(E - 1);                        // floor to a 16-byte boundary
  st.d = X - st.A;                            // the windows' misalignment, 0..E-1
  st.vb = stripe_vec<ES>(c, st, 0);
}

// Window I of the stream: 4 fp32 words, or 2 words of 2 fp16 each (loads the
// vector it needs next).
template <int ES, int I>
__device__ __forceinline__ void stripe_window(const TileCtx& c, StripeStream& st,
                                              uint32_t (&x)[ES == 4 ? 4 : 2]) {
  if constexpr (ES == 4) {
    st.va = st.vb;
    st.vb = stripe_vec<ES>(c, st, I + 1);
    const uint32_t w[8] = {st.va.x, st.va.y, st.va.z, st.va.w, st.vb.x, st.vb.y, st.vb.z, st.vb.w};
    const bool s1 = st.d & 1, s2 = st.d & 2;
    uint32_t y[6];
    static_for<0, 6>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      y[m] = s1 ? w[m + 1] : w[m];
    });
    static_for<0, 4>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      x[k] = s2 ? y[k + 2] : y[k];
    });
  } else {
    if constexpr (I % 2 == 0) {
      st.va = st.vb;
      st.vb = stripe_vec<ES>(c, st, I / 2 + 1);
    }
    // window I: half-words d + 4(I & 1) .. +3 of the 16 halves in va, vb
    const uint32_t w[8] = {st.va.x, st.va.y, st.va.z, st.va.w, st.vb.x, st.vb.y, st.vb.z, st.vb.w};
    constexpr int o = 2 * (I & 1);  // word offset of the window's pair
    const bool s4 = st.d & 4, s2 = st.d & 2;
    const uint32_t sel = (st.d & 1) ? 0x5432u : 0x3210u;
    uint32_t t[4], u[3];
    static_for<0, 4>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      t[m] = s4 ? w[o + m + 2] : w[o + m];
    });
    static_for<0, 3>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      u[m] = s2 ? t[m + 1] : t[m];
    });
    x[0] = perm_bytes(u[0], u[1], sel);
    x[1] = perm_bytes(u[1], u[2], sel);
  }
}

// Stores lane g's chunk of window I after the exchange: run q0 + 4I + g, row
// j, columns V - 4I - g .. +3, when the chunk lies inside the row and the run
// exists.  MASK: the paper-window mode (the loop ranges of Eqs. 4-9):
// elements outside p + u in [h_x, Ks-1+h_x] or q + v in [h_y, Kt-1+h_y] are
// zero.
template <int ES, int I, bool MASK>
__device__ __forceinline__ void stripe_store(const TileCtx& c, const StripePos& sp, int g,
                                             bool item_ok, uint32_t (&x)[ES == 4 ? 4 : 2]) {
  const int q = sp.q0 + 4 * I + g, vl = sp.V - 4 * I - g;
  if (!(item_ok && q < c.Ny && vl >= 0 && vl + 4 <= c.ncols)) return;
  unsigned char* p = c.out_run0 + (unsigned long long)(uint32_t)q * c.run_stride +
                     (long long)(sp.j * c.ncols + vl) * ES;
  if (MASK) {
    // element h of the chunk: p + u0 + j - h_x in [0, Ks-1], q + v0 + vl + h - h_y in [0, Kt-1]
    // (stripe tiles are odd cut-outs: no zero row or column)
    const bool row_ok = (unsigned)(sp.j - c.m1_j0) <= (unsigned)c.m1_jw;
    const int qv = q + vl - c.m1_q0;
    if constexpr (ES == 4) {
      static_for<0, 4>([&](auto hc) {
        constexpr int h = decltype(hc)::value;
        if (!row_ok || (unsigned)(qv + h) > (unsigned)c.Kt1) x[h] = 0;
      });
    } else {
      static_for<0, 2>([&](auto hc) {
        constexpr int h = decltype(hc)::value;
        const uint32_t lo = (row_ok && (unsigned)(qv + 2 * h) <= (unsigned)c.Kt1) ? 0xffffu : 0u;
        const uint32_t hm = (row_ok && (unsigned)(qv + 2 * h + 1) <= (unsigned)c.Kt1) ? 0xffff0000u : 0u;
        x[h] &= lo | hm;
      });
    }
  }
  if constexpr (ES == 4) {
    uint4 v;
    v.x = x[0];
    v.y = x[1];
    v.z = x[2];
    v.w = x[3];
    store_out16(c, p, v);
  } else {
    store_out8(c, p, x[0], x[1]);
  }
}

// Edge pass: chunks of run q that straddle a row boundary of the tile (or a
// run's ends), element by element.  Work item (q, boundary jb), jb = 0..nrows.
template <int ES, bool MASK>
__device__ __forceinline__ void stripe_edges(const TileCtx& c, int w, int nwarps, int lane,
                                             int rot) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  const int nb = c.nrows + 1;
  const int nitems = c.Ny * nb;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  for (int it = first * 32 + lane; it < nitems; it += nwarps * 32) {
    const int q = (int)fdiv((uint32_t)it, c.fnb);
    const int jb = it - q * nb;
    const int eb = jb * c.ncols;
    const int cs = eb - ((c.om0 + q + eb) & 3);  // start of the chunk holding element eb
    if (cs == eb) continue;                      // the chunk starts at the boundary
    const int e_lo = cs < 0 ? 0 : cs;
    const int e_hi = cs + 4 < c.L ? cs + 4 : c.L;
    unsigned char* orow = c.out_run0 + (unsigned long long)(uint32_t)q * c.run_stride;
    for (int e = e_lo; e < e_hi; ++e) {
      const int j = e < eb ? jb - 1 : jb;
      const int vl = e - j * c.ncols;
      const int b = (int)fmod_((uint32_t)(q + c.cb + vl), c.fNy);
      T x = smem_load_at<T>(c, c.stage_s + (uint32_t)(tab_load(c, j) + b * c.P - vl) * ES);
      if (MASK && ((unsigned)(j - c.m1_j0) > (unsigned)c.m1_jw ||
                   (unsigned)(q + vl - c.m1_q0) > (unsigned)c.Kt1))
        x = 0;
      store_out(c, reinterpret_cast<T*>(orow) + e, x);
    }
  }
}

#ifndef LFBP_HOST_EMULATION
// The 4 x 4 exchange of one window (all 32 lanes take part).
template <int ES>
__device__ __forceinline__ void stripe_exchange(uint32_t (&x)[ES == 4 ? 4 : 2], int g) {
  if constexpr (ES == 4) {
    uint32_t s[2], r[2];
    xs_a32(x, g, s);
    r[0] = __shfl_xor_sync(0xffffffffu, s[0], 2);
    r[1] = __shfl_xor_sync(0xffffffffu, s[1], 2);
    xr_a32(x, g, r);
    xs_b32(x, g, s);
    r[0] = __shfl_xor_sync(0xffffffffu, s[0], 1);
    r[1] = __shfl_xor_sync(0xffffffffu, s[1], 1);
    xr_b32(x, g, r);
  } else {
    uint32_t r = __shfl_xor_sync(0xffffffffu, xs_a16(x, g), 2);
    xr_a16(x, g, r);
    r = __shfl_xor_sync(0xffffffffu, xs_b16(x, g), 1);
    xr_b16(x, g, r);
  }
}

// Consumer side, stripe path.  Warp step u covers stripes 8u .. 8u+7 (lanes
// 4s .. 4s+3 take stripe 8u+s); every lane of the warp runs every step, so the
// exchanges see all 32 lanes.  The windows of a stripe are cut out, exchanged
// and stored one after the other, which keeps few of them in registers.
// Then the edge pass.
template <int ES, int S, bool MASK>
__device__ __forceinline__ void gather_stripes(const TileCtx& c, int w, int nwarps, int lane,
                                               int rot) {
  const int g = lane & 3, gs = lane >> 2;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  for (int u = first; u < c.nsteps_s; u += nwarps) {
    int item = u * 8 + gs;
    const bool ok = item < c.nitems_s;
    if (!ok) item = c.nitems_s - 1;  // a valid position; nothing is stored
    const StripePos sp = stripe_pos<S>(c, item);
    StripeStream st;
    stripe_begin<ES>(c, sp, g, st);
    static_for<0, S>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      uint32_t x[ES == 4 ? 4 : 2];
      stripe_window<ES, i>(c, st, x);
      stripe_exchange<ES>(x, g);
      stripe_store<ES, i, MASK>(c, sp, g, ok, x);
    });
  }
  stripe_edges<ES, MASK>(c, w, nwarps, lane, rot);
}

template <int ES, bool MASK>
__device__ __forceinline__ void gather_stripes_s(const TileCtx& c, int w, int nwarps, int lane,
                                                 int rot) {
  switch (c.S) {
    case 1: gather_stripes<ES, 1, MASK>(c, w, nwarps, lane, rot); break;
    case 2: gather_stripes<ES, 2, MASK>(c, w, nwarps, lane, rot); break;
    case 3: gather_stripes<ES, 3, MASK>(c, w, nwarps, lane, rot); break;
#if LFBP_STRIPE_SMAX >= 4
    case 4: gather_stripes<ES, 4, MASK>(c, w, nwarps, lane, rot); break;
#endif
#if LFBP_STRIPE_SMAX >= 5
    case 5: gather_stripes<ES, 5, MASK>(c, w, nwarps, lane, rot); break;
#endif
    default: break;
  }
}

// Consumer side of a stripe tile (c.stripe).
__device__ __forceinline__ void gather_stripes_ctx(const TileCtx& cs, int w, int nwarps, int lane,
                                                   int rot) {
  const TileCtx c = cs;  // into registers, once per tile
  if (c.es == 4) {
    if (c.mode == 0)
      gather_stripes_s<4, false>(c, w, nwarps, lane, rot);
    else
      gather_stripes_s<4, true>(c, w, nwarps, lane, rot);
  } else {
    if (c.mode == 0)
      gather_stripes_s<2, false>(c, w, nwarps, lane, rot);
    else
      gather_stripes_s<2, true>(c, w, nwarps, lane, rot);
  }
}
#endif

}  // namespace lfbp
