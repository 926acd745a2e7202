// Device building blocks of the H -> H' gather (sm_103a).
//
// The map of one depth (Sec. 3, Eqs. 4-9, as a full permutation):
//     H'[p][q][u][v] = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]
// factorises into a row part acting on (a, s) and a column part acting on
// (b, t).  An output "row" (p, u) is Ny runs of Kt contiguous elements (one
// per q, stride Ks*Kt); its source row (a, s) = ((p+u-c_s) mod Nx, Ks-1-u) is
// Ny contiguous segments of Kt elements (one per b).  Within the row, output
// element (q, v) comes from segment b = (q+v-c_t) mod Ny at t = Kt-1-v: a
// reversal of the pixel axis and a cyclic exchange of the cell axis.
//
// A tile is `nrows` consecutive output rows u0..u0+nrows-1 of one p (and a
// column range v0..v0+ncols-1, all of Kt unless a row is too large for one
// stage).  Its output is Ny contiguous runs of nrows*ncols elements; its
// input is nrows*Ny segments, loaded with TMA bulk copies into shared memory
// (each widened to 16-byte boundaries, since segments start anywhere), then
// gathered through the index map and written with 128-bit stores.
#pragma once
#include <cstdint>
#include <type_traits>

namespace lfbp {

constexpr int kMaxBatch = 64;       // arrays per batched launch
constexpr int kStatusTimeout = -7;  // LFBP_ERR_TIMEOUT

// One (array, depth) of a batched launch.
struct JobDesc {
  unsigned long long off_bytes;  // byte offset of the depth inside its array
  int arr;                       // array slot in BatchPtrs
  int Nx, Ny, Ks, Kt;
  int es;    // bytes per element: 4 or 2
  int mode;  // 0 transpose, 1 paper window (forward), 2 paper window (adjoint)
  int pad;
};
static_assert(sizeof(JobDesc) == 40, "JobDesc layout");

// One tile of a job.
struct TileDesc {
  unsigned job;
  unsigned short p, u0, v0, nrows, ncols, pad;
};
static_assert(sizeof(TileDesc) == 16, "TileDesc layout");

struct BatchPtrs {
  const unsigned char* in[kMaxBatch];
  unsigned char* out[kMaxBatch];
  unsigned long long in_bytes[kMaxBatch];
};

// Exact n / d for n, d < 2^16 via one multiply-high (d is tile-uniform).
struct FastDiv {
  uint32_t d, m;
};
__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.m = d > 1 ? (uint32_t)((0x100000000ull + d - 1) / d) : 0u;
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) {
  return f.d == 1 ? n : __umulhi(n, f.m);
}
__device__ __forceinline__ uint32_t fmod_(uint32_t n, FastDiv f) { return n - fdiv(n, f) * f.d; }

// Bytes of the shared-memory slot that holds a segment of n elements widened
// to 16-byte boundaries, whatever its alignment.
__host__ __device__ inline uint32_t slot_bytes(uint32_t n, uint32_t es) {
  return (n * es + 16u - es + 15u) & ~15u;
}

inline int lfbp_min(int a, int b) { return a < b ? a : b; }
inline int lfbp_max(int a, int b) { return a > b ? a : b; }

// Host side: tiling of one depth, target = shared-memory bytes of one tile.
// Tiling of one depth: rows per tile J, columns per tile V (V = Kt unless one
// row does not fit the target), and the counts of u- and v-blocks.
struct DepthTiling {
  int J, V, nU, nV;
  int max_tile_bytes;
};

inline DepthTiling tile_depth(int Ny, int Ks, int Kt, int es, int target) {
  DepthTiling d;
  const int row = Ny * (int)slot_bytes(Kt, es);
  if (row <= target) {
    d.V = Kt;
    d.nV = 1;
    int J = lfbp_max(1, lfbp_min(Ks, target / row));
    d.nU = (Ks + J - 1) / J;
    d.J = (Ks + d.nU - 1) / d.nU;
    d.max_tile_bytes = d.J * row;
  } else {
    d.J = 1;
    d.nU = Ks;
    int nV = (row + target - 1) / target;
    for (;; ++nV) {
      const int V = (Kt + nV - 1) / nV;
      if (Ny * (int)slot_bytes(V, es) <= target || V == 1) break;
    }
    d.V = (Kt + nV - 1) / nV;
    d.nV = (Kt + d.V - 1) / d.V;
    d.max_tile_bytes = Ny * (int)slot_bytes(d.V, es);
  }
  return d;
}

// Everything the consumers need about the tile in a stage (filled by the
// producer lane, read by all consumer threads).
struct TileInfo {
  unsigned long long out_run0;    // byte address of output run q = 0, element v0 of row u0
  unsigned long long run_stride;  // bytes between runs q and q+1 (Ks*Kt*es)
  int tile;                       // tile index, < 0 = no more work
  int es, mode;
  int Nx, Ny, Ks, Kt;
  int p, u0, v0, nrows, ncols;
  int L;       // elements per output run = nrows*ncols
  int NC;      // 16-byte chunks reserved per run (covers any misalignment)
  int slote;   // slot pitch in elements
  int ap0;     // (p + u0 - c_s) mod Nx: source cell position of row u0
  int s0;      // Ks - 1 - u0: source pixel row of row u0
  int cb;      // (v0 - c_t) mod Ny
  int om0;     // misalignment (elements mod 16/es) of output run q = 0
  int kk;      // (Ks*Kt) mod (16/es): misalignment step between q runs / b segments
  int inm;     // misalignment of the input depth base + t_lo (elements mod 16/es)
  int nkk;     // (Ny*Ks*Kt) mod (16/es)
  int ktm;     // Kt mod (16/es)
  FastDiv fNC, fncols, fNy, fNx;
};

// ---------------------------------------------------------------- PTX ----
// Under LFBP_HOST_EMULATION the including translation unit supplies host
// stand-ins for these primitives (and for the two global-store helpers and
// the shared-memory index check below), so that the tile code of this header
// can be run on the CPU with every memory access checked.
#ifndef LFBP_HOST_EMULATION
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up after `limit_ns` of wall time
// (or when *abort is raised by another thread of the CTA), then returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  const volatile int* abort, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
    if ((it & 63u) == 63u) {
      if (globaltimer_ns() - t0 > limit_ns) return false;
      __nanosleep(64);
    }
  }
  return false;
}

__device__ __forceinline__ void st_global_16(void* p, uint4 w) {
  *reinterpret_cast<uint4*>(p) = w;
}
template <class T>
__device__ __forceinline__ void st_global_elem(T* p, T v) {
  *p = v;
}
#define LFBP_SMEM_CHECK(idx)
#endif  // LFBP_HOST_EMULATION

__device__ __forceinline__ int pos_mod(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// Producer side: fill `ti` for tile `td` of job `jd` (one thread).
__device__ __forceinline__ void make_tile_info(TileInfo& ti, int tile, const TileDesc& td,
                                               const JobDesc& jd, const unsigned char* in_depth,
                                               unsigned char* out_depth) {
  const int es = jd.es, E = 16 / es;
  ti.tile = tile;
  ti.es = es;
  ti.mode = jd.mode;
  ti.Nx = jd.Nx;
  ti.Ny = jd.Ny;
  ti.Ks = jd.Ks;
  ti.Kt = jd.Kt;
  ti.p = td.p;
  ti.u0 = td.u0;
  ti.v0 = td.v0;
  ti.nrows = td.nrows;
  ti.ncols = td.ncols;
  ti.L = td.nrows * td.ncols;
  ti.NC = (E - 1 + ti.L + E - 1) / E;
  ti.slote = (int)(slot_bytes(td.ncols, es) / es);
  const int cs = (jd.Ks - 1) / 2, ct = (jd.Kt - 1) / 2;
  ti.ap0 = pos_mod(td.p + td.u0 - cs, jd.Nx);
  ti.s0 = jd.Ks - 1 - td.u0;
  ti.cb = pos_mod(td.v0 - ct, jd.Ny);
  const unsigned long long KK = (unsigned long long)jd.Ks * (unsigned long long)jd.Kt;
  const unsigned long long run0 =
      ((unsigned long long)td.p * jd.Ny * jd.Ks + td.u0) * jd.Kt + td.v0;  // elements
  const unsigned long long out0 = (unsigned long long)out_depth + run0 * es;
  ti.out_run0 = out0;
  ti.run_stride = KK * es;
  ti.om0 = (int)((out0 / es) & (E - 1));
  ti.kk = (int)(KK & (E - 1));
  const int t_lo = jd.Kt - td.v0 - td.ncols;
  ti.inm = (int)((((unsigned long long)in_depth / es) + t_lo) & (E - 1));
  ti.nkk = (int)(((unsigned long long)jd.Ny * KK) & (E - 1));
  ti.ktm = jd.Kt & (E - 1);
  ti.fNC = make_fastdiv(ti.NC);
  ti.fncols = make_fastdiv(td.ncols);
  ti.fNy = make_fastdiv(jd.Ny);
  ti.fNx = make_fastdiv(jd.Nx);
}

// Producer side: issue the bulk copies of the tile's input segments into the
// stage.  Called by all 32 lanes of one warp; lane 0 arrives on `bar` after
// every lane has registered its bytes and issued its copies.  The last <16
// bytes of an array that a 16-byte-widened copy would over-read are copied
// with ordinary loads instead.
__device__ __forceinline__ void issue_tile_loads(const TileDesc& td, const JobDesc& jd,
                                                 const unsigned char* in_depth,
                                                 const unsigned char* in_safe_end,
                                                 unsigned char* stage, uint32_t bar, int lane) {
  const int es = jd.es;
  const int Ny = jd.Ny, Ks = jd.Ks, Kt = jd.Kt;
  const int nslots = td.nrows * Ny;
  const uint32_t sb = slot_bytes(td.ncols, es);
  const int cs = (Ks - 1) / 2;
  const int t_lo = Kt - td.v0 - td.ncols;
  const uint32_t seg_bytes = (uint32_t)td.ncols * es;
  // pass 1: bytes this lane will bring in with bulk copies
  uint32_t my_bytes = 0;
  for (int i = lane; i < nslots; i += 32) {
    const int j = i / Ny, b = i - j * Ny;
    const int a = pos_mod(td.p + td.u0 + j - cs, jd.Nx);
    const int s = Ks - 1 - td.u0 - j;
    const unsigned long long seg = (((unsigned long long)a * Ny + b) * Ks + s) * Kt + t_lo;
    const unsigned char* src = in_depth + seg * es;
    const uintptr_t lo = (uintptr_t)src & ~(uintptr_t)15;
    uintptr_t hi = ((uintptr_t)src + seg_bytes + 15) & ~(uintptr_t)15;
    if (hi > (uintptr_t)in_safe_end) hi = (uintptr_t)in_safe_end;
    if (hi > lo) my_bytes += (uint32_t)(hi - lo);
  }
  if (my_bytes) mbar_expect_tx(bar, my_bytes);
  bool fixed = false;
  for (int i = lane; i < nslots; i += 32) {
    const int j = i / Ny, b = i - j * Ny;
    const int a = pos_mod(td.p + td.u0 + j - cs, jd.Nx);
    const int s = Ks - 1 - td.u0 - j;
    const unsigned long long seg = (((unsigned long long)a * Ny + b) * Ks + s) * Kt + t_lo;
    const unsigned char* src = in_depth + seg * es;
    const uintptr_t lo = (uintptr_t)src & ~(uintptr_t)15;
    const uintptr_t end = (uintptr_t)src + seg_bytes;
    uintptr_t hi = (end + 15) & ~(uintptr_t)15;
    unsigned char* dst = stage + (size_t)i * sb;
    if (hi > (uintptr_t)in_safe_end) {
      hi = (uintptr_t)in_safe_end > lo ? (uintptr_t)in_safe_end : lo;
      // tail beyond the last full 16-byte block of the array: plain loads
      for (uintptr_t x = hi > (uintptr_t)src ? hi : (uintptr_t)src; x < end; x += es) {
        if (es == 4)
          *(uint32_t*)(dst + (x - lo)) = __ldg((const unsigned int*)x);
        else
          *(uint16_t*)(dst + (x - lo)) = __ldg((const unsigned short*)x);
      }
      fixed = true;
    }
    if (hi > lo) bulk_g2s(smem_addr(dst), (const void*)lo, (uint32_t)(hi - lo), bar);
  }
  if (fixed) fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}

// Consumer side: gather the tile from the stage through the index map and
// write its Ny output runs with 16-byte stores.  Threads [tid0, tid0+nthr)
// share the work; chunk g = (run q, 16-byte block k of that run).
template <int ES, int MODE>
__device__ __forceinline__ void gather_store_tile(const TileInfo& ti, const unsigned char* stage,
                                                  int tid, int nthr) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  constexpr int E = 16 / ES;
  const T* sm = reinterpret_cast<const T*>(stage);
  const int Ny = ti.Ny, Nx = ti.Nx, L = ti.L, NC = ti.NC, ncols = ti.ncols, slote = ti.slote;
  const int kk = ti.kk, inm = ti.inm, nkk = ti.nkk, ktm = ti.ktm, s0 = ti.s0;
  const int hx = (Nx - 1) / 2, hy = (Ny - 1) / 2;
  const int total = Ny * NC;
  for (int g = tid; g < total; g += nthr) {
    const int q = (int)fdiv((uint32_t)g, ti.fNC);
    const int k = g - q * NC;
    const int m = (ti.om0 + q * kk) & (E - 1);
    const int e0 = k * E - m;
    if (e0 >= L) continue;
    unsigned char* out = reinterpret_cast<unsigned char*>(ti.out_run0 + (unsigned long long)q * ti.run_stride) +
                         (long long)e0 * ES;
    const int ef = e0 > 0 ? e0 : 0;
    int j = (int)fdiv((uint32_t)ef, ti.fncols);
    int vl = ef - j * ncols;
    int a = (int)fmod_((uint32_t)(ti.ap0 + j), ti.fNx);
    int mj = (inm + a * nkk + (s0 - j) * ktm) & (E - 1);
    const int bq0 = (int)fmod_((uint32_t)(q + ti.cb), ti.fNy);
    int b = (int)fmod_((uint32_t)(bq0 + vl), ti.fNy);
    bool rowkeep = true;
    if (MODE == 1) rowkeep = (ti.p + ti.u0 + j >= hx) && (ti.p + ti.u0 + j <= ti.Ks - 1 + hx);
    if (MODE == 2) rowkeep = (a + s0 - j >= hx) && (a + s0 - j <= ti.Ks - 1 + hx);
    T vals[E];
    uint32_t valid = 0;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int e = e0 + i;
      vals[i] = 0;
      if (e >= 0 && e < L) {
        valid |= 1u << i;
        const int idx = (j * Ny + b) * slote + ((mj + b * kk) & (E - 1)) + ncols - 1 - vl;
        LFBP_SMEM_CHECK(idx);
        T x = sm[idx];
        if (MODE == 1) {
          const int v = ti.v0 + vl;
          const bool keep = rowkeep && (q + v >= hy) && (q + v <= ti.Kt - 1 + hy);
          x = keep ? x : (T)0;
        } else if (MODE == 2) {
          const int t = ti.Kt - 1 - ti.v0 - vl;
          const bool keep = rowkeep && (b + t >= hy) && (b + t <= ti.Kt - 1 + hy);
          x = keep ? x : (T)0;
        }
        vals[i] = x;
        ++vl;
        ++b;
        if (b == Ny) b = 0;
        if (vl == ncols) {
          vl = 0;
          ++j;
          ++a;
          if (a == Nx) a = 0;
          mj = (inm + a * nkk + (s0 - j) * ktm) & (E - 1);
          b = bq0;
          if (MODE == 1) rowkeep = (ti.p + ti.u0 + j >= hx) && (ti.p + ti.u0 + j <= ti.Ks - 1 + hx);
          if (MODE == 2) rowkeep = (a + s0 - j >= hx) && (a + s0 - j <= ti.Ks - 1 + hx);
        }
      }
    }
    if (valid == (1u << E) - 1u) {
      uint4 w;
      if (ES == 4) {
        w.x = vals[0]; w.y = vals[1]; w.z = vals[2]; w.w = vals[3];
      } else {
        w.x = (uint32_t)vals[0] | ((uint32_t)vals[1] << 16);
        w.y = (uint32_t)vals[2] | ((uint32_t)vals[3] << 16);
        w.z = (uint32_t)vals[4] | ((uint32_t)vals[5] << 16);
        w.w = (uint32_t)vals[6] | ((uint32_t)vals[7] << 16);
      }
      st_global_16(out, w);
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i)
        if (valid & (1u << i)) st_global_elem(reinterpret_cast<T*>(out) + i, vals[i]);
    }
  }
}

template <int MODE>
__device__ __forceinline__ void gather_store_any(const TileInfo& ti, const unsigned char* stage,
                                                 int tid, int nthr) {
  if (ti.es == 4)
    gather_store_tile<4, MODE>(ti, stage, tid, nthr);
  else
    gather_store_tile<2, MODE>(ti, stage, tid, nthr);
}

__device__ __forceinline__ void gather_store_dispatch(const TileInfo& ti, const unsigned char* stage,
                                                      int tid, int nthr) {
  if (ti.mode == 0)
    gather_store_any<0>(ti, stage, tid, nthr);
  else if (ti.mode == 1)
    gather_store_any<1>(ti, stage, tid, nthr);
  else
    gather_store_any<2>(ti, stage, tid, nthr);
}

}  // namespace lfbp
