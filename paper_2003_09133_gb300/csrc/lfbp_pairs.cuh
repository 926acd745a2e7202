// Pair gather: the consumer of the H -> H' map (transpose mode) for tiles
// whose run stride Ks*Kt is 1 modulo the chunk length E = 16/es (every odd
// square cut-out, among others).
//
// In tile row j, output element (q, vl) of run q is read from stage element
//     idx(q, vl) = rb_j + b*P - vl,   b = (q + cb + vl) mod Ny,
// and its anti-diagonal neighbour (q+1, vl-1) from the same segment b one
// element further on, idx + 1 (Eqs. 5 and 8: the cell index moves with the
// pixel index, and the pixel axis is reversed).  So when idx is even one
// aligned two-element load (8 bytes in fp32, 4 in fp16) brings an element of
// run q and one of run q+1.
//
// PAIR UNIT.  All runs on one anti-diagonal D = q + vl of row j start their
// chunk in the same segment b_D = (cb + D) mod Ny.  Along a chunk (columns
// vl .. vl+E-1 of run q) the index steps by P - 1, which is even (P = Ks*Kt =
// 1 mod E), except where the segment wraps from Ny-1 to 0 (at element
// kw = Ny - b_D), where it also drops by W = Ny*P, which is odd (Ny, P odd).
// On the anti-diagonal, idx(q, D - q) = rb_j + b_D*P - D + q, so the runs q
// with even idx are every other run, q = pi, pi+2, ..., pi = (rb_j + b_D*P - D)
// mod 2.  A unit is the pair (q, q+1) of such a run and its successor: the
// chunk of run q at vl and the chunk of run q+1 at vl-1.  Because Ks*Kt = 1
// (mod E) both chunks are 16-byte aligned in the output.  Elements k < kw of
// the unit come from one aligned two-element load each; elements k >= kw sit
// at odd indexes and take two loads (the element of run q is the upper half of
// the pair below, the element of run q+1 the lower half of the pair above).
//
// COVERAGE.  Chunks wholly inside one tile row and inside the run are either
// in a unit whose two chunks are both whole (pair pass) or not (at most two per
// anti-diagonal, at its ends: the rest pass, one chunk each).  Chunks that
// contain a row boundary or a run end are stored element by element (edge
// pass).
#pragma once

namespace lfbp {

// two consecutive stage elements at an index that is a multiple of two
template <int ES>
struct Pair2;
template <>
struct Pair2<4> {
  using T = uint2;
};
template <>
struct Pair2<2> {
  using T = uint32_t;
};

template <int ES>
__device__ __forceinline__ typename Pair2<ES>::T lds_pair(const TileCtx& c, uint32_t addr) {
#if LFBP_CHECKED
  const long long rel = (long long)addr - (long long)c.stage_s;
  if (rel < 0 || rel + 2 * ES > c.tile_bytes || (rel & (2 * ES - 1))) {
    check_fail(1, rel, c.tile_bytes);
    return typename Pair2<ES>::T{};
  }
#endif
  (void)c;
  if constexpr (ES == 4)
    return lds64(addr);
  else
    return lds<uint32_t>(addr);
}

// The element pair (run q, run q+1) of unit element k >= kw: the upper
// element of the pair at idx - 1 and the lower element of the pair at idx + 1.
__device__ __forceinline__ uint2 pair_join(uint2 lo, uint2 hi) { return make_uint2(lo.y, hi.x); }
__device__ __forceinline__ uint32_t pair_join(uint32_t lo, uint32_t hi) {
  return perm_bytes(lo, hi, 0x5432u);
}

// Stores the two chunks of a unit: run q's elements are the lower halves of
// the pairs, run q+1's the upper halves.
__device__ __forceinline__ void pair_store(const TileCtx& c, unsigned char* pq, unsigned char* pq1,
                                           const uint2 (&x)[4]) {
  store_out16(c, pq, make_uint4(x[0].x, x[1].x, x[2].x, x[3].x));
  store_out16(c, pq1, make_uint4(x[0].y, x[1].y, x[2].y, x[3].y));
}
__device__ __forceinline__ void pair_store(const TileCtx& c, unsigned char* pq, unsigned char* pq1,
                                           const uint32_t (&x)[8]) {
  uint4 a, b;
  a.x = perm_bytes(x[0], x[1], 0x5410u);
  a.y = perm_bytes(x[2], x[3], 0x5410u);
  a.z = perm_bytes(x[4], x[5], 0x5410u);
  a.w = perm_bytes(x[6], x[7], 0x5410u);
  b.x = perm_bytes(x[0], x[1], 0x7632u);
  b.y = perm_bytes(x[2], x[3], 0x7632u);
  b.z = perm_bytes(x[4], x[5], 0x7632u);
  b.w = perm_bytes(x[6], x[7], 0x7632u);
  store_out16(c, pq, a);
  store_out16(c, pq1, b);
}

// Position of anti-diagonal d of row j: D, its segment b_D, the row base and
// the first run of the row's pairs (pi).
struct PairDiag {
  int D, bD, rb, pi;
};

template <int ES>
__device__ __forceinline__ PairDiag pair_diag(const TileCtx& c, int j, int d) {
  constexpr int E = 16 / ES;
  PairDiag g;
  const int o = (c.om0 + j * c.ncols) & (E - 1);  // run 0's chunks start at vl = -o (mod E)
  g.D = E * d - o;
  g.bD = (int)fmod2((uint32_t)(c.cbb + g.D), c.fNy);
  g.rb = tab_load(c, j);
  g.pi = (g.rb + g.bD * c.P - g.D) & 1;
  return g;
}

// Output address of element e of run q.
__device__ __forceinline__ unsigned char* run_elem(const TileCtx& c, int q, int e) {
  return c.out_run0 + (unsigned long long)(uint32_t)q * c.run_stride + (long long)e * c.es;
}

// The pair pass.  Unit u = ((j * npr + r) * nu + i): row j, pair slot r
// (runs pi + 2r, pi + 2r + 1), and the i-th anti-diagonal on which slot r can
// hold two whole chunks: D in [2r + 1, 2r + 1 + ncols - E], i.e. d from
// ceil((2r + 1 + o_j) / E) on (nu of them cover that range).  Lanes take
// consecutive anti-diagonals, so the chunks a warp stores lie along few runs.
template <int ES>
__device__ __forceinline__ void gather_pair_units(const TileCtx& c, int w, int nwarps, int lane,
                                                  int rot) {
  constexpr int E = 16 / ES;
  using P2 = typename Pair2<ES>::T;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  for (int u = first * 32 + lane; u < c.punits; u += nwarps * 32) {
    const int jr = (int)fdiv2((uint32_t)u, c.fpnu);
    const int i = u - jr * c.pnu;
    const int j = (int)fdiv((uint32_t)jr, c.fpnpr);
    const int r = jr - j * c.pnpr;
    const int o = (c.om0 + j * c.ncols) & (E - 1);
    const int d = (2 * r + o + E) / E + i;  // ceil((2r + 1 + o) / E) + i
    const PairDiag g = pair_diag<ES>(c, j, d);
    const int q = g.pi + 2 * r;
    const int vl = g.D - q;
    // both chunks whole inside the row: run q at [vl, vl+E), run q+1 at [vl-1, vl-1+E)
    if (q + 1 >= c.Ny || vl < 1 || vl + E > c.ncols) continue;
    const int kw = c.Ny - g.bD;
    const uint32_t A = c.stage_s + (uint32_t)(g.rb + g.bD * c.P - vl) * ES;
    P2 x[E];
    static_for<0, E>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const uint32_t a = A + (uint32_t)k * c.D;
      if (k < kw) {
        x[k] = lds_pair<ES>(c, a);
      } else {
        const uint32_t aw = a - c.W;  // the element's odd index after the wrap
        x[k] = pair_join(lds_pair<ES>(c, aw - ES), lds_pair<ES>(c, aw + ES));
      }
    });
    const int e = j * c.ncols + vl;
    pair_store(c, run_elem(c, q, e), run_elem(c, q + 1, e - 1), x);
  }
}

// The rest pass: per anti-diagonal, the chunk at its lower end (run qa, when
// its partner qa - 1 lies outside the row) and at its upper end (run qb, when
// its partner qb + 1 does), one chunk each.  Item i = (j * nd + d) * 2 + side.
template <int ES>
__device__ __forceinline__ void gather_pair_rest(const TileCtx& c, int w, int nwarps, int lane,
                                                 int rot) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  constexpr int E = 16 / ES;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  const int nitems = c.nrows * c.pnd * 2;
  for (int i = first * 32 + lane; i < nitems; i += nwarps * 32) {
    const int jd = i >> 1, side = i & 1;
    const int j = (int)fdiv2((uint32_t)jd, c.fpnd);
    const int d = jd - j * c.pnd;
    const PairDiag g = pair_diag<ES>(c, j, d);
    // runs with a whole chunk on this anti-diagonal: vl = D - q in [0, ncols - E]
    const int qa = g.D - (c.ncols - E) > 0 ? g.D - (c.ncols - E) : 0;
    const int qb = g.D < c.Ny - 1 ? g.D : c.Ny - 1;
    if (qa > qb) continue;
    // a run q is paired upwards when q = pi (mod 2), downwards otherwise
    const int q = side ? qb : qa;
    const bool up = ((q - g.pi) & 1) == 0;
    const bool partner_ok = up ? q + 1 <= qb : q - 1 >= qa;
    if (partner_ok) continue;
    if (side == 1 && qa == qb) continue;  // one chunk only: the lower side takes it
    const int vl = g.D - q;
    const int kw = c.Ny - g.bD;
    const uint32_t A = c.stage_s + (uint32_t)(g.rb + g.bD * c.P - vl) * ES;
    T v[E];
    static_for<0, E>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      uint32_t a = A + (uint32_t)k * c.D;
      if (k >= kw) a -= c.W;
      v[k] = smem_load_at<T>(c, a);
    });
    store_out16(c, run_elem(c, q, j * c.ncols + vl), pack16(v));
  }
}

// The edge pass: chunks of run q that contain a row boundary of the tile or a
// run end.  Item (q, jb), jb = 0..nrows: the chunk that holds element
// jb * ncols (for jb = nrows, the run's last partial chunk).  A chunk across
// an inner row boundary lies inside the run: it is gathered with the chunk
// path's two-row addressing and stored whole; the chunks cut by the run's
// ends go element by element.
template <int ES>
__device__ __forceinline__ void gather_pair_edges(const TileCtx& c, int w, int nwarps, int lane,
                                                  int rot) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  constexpr int E = 16 / ES;
  const int nb = c.nrows + 1;
  const int nitems = c.Ny * nb;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  for (int it = first * 32 + lane; it < nitems; it += nwarps * 32) {
    const int q = (int)fdiv((uint32_t)it, c.fnb);
    const int jb = it - q * nb;
    const int eb = jb * c.ncols;
    const int cs = eb - ((c.om0 + q + eb) & (E - 1));  // start of the chunk holding element eb
    if (cs == eb) continue;                            // the chunk starts at the boundary
    if (cs >= 0 && cs + E <= c.L) {                    // inside the run: across rows jb-1, jb
      const ChunkAddr s = chunk_addr<ES, false>(c, q, cs);
      T v[E];
      static_for<0, E>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = smem_load_at<T>(c, chunk_elem<false>(c, s, k));
      });
      store_out16(c, run_elem(c, q, cs), pack16(v));
      continue;
    }
    const int e_lo = cs < 0 ? 0 : cs;
    const int e_hi = cs + E < c.L ? cs + E : c.L;
    for (int e = e_lo; e < e_hi; ++e) {
      const int j = e < eb ? jb - 1 : jb;
      const int vl = e - j * c.ncols;
      const int b = (int)fmod_((uint32_t)(q + c.cb + vl), c.fNy);
      const T x = smem_load_at<T>(c, c.stage_s + (uint32_t)(tab_load(c, j) + b * c.P - vl) * ES);
      store_out(c, reinterpret_cast<T*>(run_elem(c, q, e)), x);
    }
  }
}

template <int ES>
__device__ __forceinline__ void gather_pairs(const TileCtx& c, int w, int nwarps, int lane,
                                             int rot) {
  gather_pair_units<ES>(c, w, nwarps, lane, rot);
  gather_pair_rest<ES>(c, w, nwarps, lane, rot);
  gather_pair_edges<ES>(c, w, nwarps, lane, rot);
}

// Consumer side of a pair tile (c.pair).
__device__ __forceinline__ void gather_pairs_ctx(const TileCtx& cs, int w, int nwarps, int lane,
                                                 int rot) {
  const TileCtx c = cs;  // into registers, once per tile
  if (c.es == 4)
    gather_pairs<4>(c, w, nwarps, lane, rot);
  else
    gather_pairs<2>(c, w, nwarps, lane, rot);
}

}  // namespace lfbp
