// Device building blocks of the H -> H' gather (sm_103a).
//
// The map of one depth (Sec. 4, Eqs. 4-9, as a full permutation):
//     H'[p][q][u][v] = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]
// factorises into a row part acting on (a, s) and a column part acting on
// (b, t).  An output "row" (p, u) is Ny runs of Kt contiguous elements (one
// per q, stride Ks*Kt); its source row (a, s) = ((p+u-c_s) mod Nx, Ks-1-u) is
// Ny contiguous segments of Kt elements (one per b).  Within the row, output
// element (q, v) comes from segment b = (q+v-c_t) mod Ny at t = Kt-1-v: a
// reversal of the pixel axis and a cyclic exchange of the cell axis, i.e. a
// walk along a diagonal of the (b, t) plane.
//
// TILE.  `nrows` consecutive output rows u0.. of one p, and the column range
// v0..v0+ncols-1 (all of Kt unless one row does not fit a stage; then
// nrows = 1).  Its output is Ny contiguous runs of nrows*ncols elements (one
// per q); its input is nrows*Ny segments of ncols elements.
//
// SHARED-MEMORY LAYOUT.  Segment (j, b) is brought in by one TMA bulk copy,
// widened to 16-byte boundaries because segments start anywhere; its element
// i lands at  j*RP + R_j + b*P + i  (elements), where the slot pitch P is
// congruent to Ks*Kt modulo 16/esize and R_j is the 16-byte phase of segment
// (j, 0).  Every copy destination is then 16-byte aligned, and the address of
// a diagonal walk is linear in b.  Among the pitches allowed, the planner
// picks the one with the fewest shared-memory bank conflicts for the gather's
// access pattern (choose_pitch).
//
// GATHER.  The output runs of a tile are cut into aligned 128-byte lines; a
// consumer warp step covers 4 consecutive lines (of one run, or straddling
// two), each lane one 16-byte chunk: 4 fp32 or 8 fp16 consecutive output
// elements, written with one 16-byte store.  Inside a row, consecutive output
// elements are diagonal neighbours (b+1, t-1) in the stage, one slot pitch
// minus one element apart, so a chunk's shared-memory addresses follow from
// its first one by adding that stride, corrected where the chunk wraps from
// segment Ny-1 to 0 or crosses into the next row (branch-free selects).
#pragma once
#include <cstdint>
#include <type_traits>

namespace lfbp {

constexpr int kMaxBatch = 64;       // arrays per batched launch
constexpr int kStatusTimeout = -7;  // LFBP_ERR_TIMEOUT
constexpr int kGroupsPerItem = 4;   // 128-byte groups per run handled by one consumer work item
                                    // (element-walk path)
constexpr int kMaxTileRows = 64;    // rows per tile (bounds the per-tile row-base table)
// One-row tiles whose runs are at least this long store the chunks cut by a
// run's ends inside the main loop; shorter ones leave them to the edge pass
// (measured: runs of 616 B, N = 51: 3827 -> 4575 GB/s with the edge pass;
// 2028 B, N = 11, K = 507: 6080 -> 6007).
constexpr int kInlineEndsBytes = 1800;

// One tile, self-contained (32 bytes).
struct TileDesc {
  unsigned long long off_bytes;  // byte offset of the depth inside its array
  unsigned short p, u0, v0, nrows, ncols;
  unsigned short Nx, Ny, Ks, Kt;
  unsigned short P;     // slot pitch in elements
  unsigned char arr;    // array slot in BatchPtrs
  unsigned char flags;  // bit 0: fp16 storage; bits 1-2: mode; bits 3-4: Ks, Kt even;
                        // bit 5: the pair consumer is off for this tile
  unsigned short shape; // index of the tile's TileShape in the launch's shape table
};
static_assert(sizeof(TileDesc) == 32, "TileDesc layout");

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
  f.m = d > 1 ? 0xffffffffu / d + 1u : 0u;  // ceil(2^32 / d)
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) {
  return f.d == 1 ? n : __umulhi(n, f.m);
}
__device__ __forceinline__ uint32_t fmod_(uint32_t n, FastDiv f) { return n - fdiv(n, f) * f.d; }

inline int lfbp_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int lfbp_dmin(int a, int b) { return a < b ? a : b; }
inline int lfbp_max(int a, int b) { return a > b ? a : b; }

#ifndef LFBP_STRIPE_SMAX
#define LFBP_STRIPE_SMAX 5
#endif
#ifndef LFBP_STRIPES
#define LFBP_STRIPES 1  // 0: every tile takes the chunk or element-walk path
#endif
constexpr int kStripeMaxS = LFBP_STRIPE_SMAX;  // run blocks per stripe (template instances 1..)
#ifndef LFBP_PAIRS
#define LFBP_PAIRS 1  // 0: no tile takes the pair path
#endif
constexpr bool kPairs = LFBP_PAIRS != 0;

// Run blocks per stripe for nrb = ceil(Ny/4) run blocks: all of them up to
// five; beyond, the size in 3..5 whose bands waste the fewest chunk slots
// (ties: the larger).
__host__ __device__ inline int stripe_S(int nrb) {
  if (nrb <= kStripeMaxS) return nrb;
  int best = kStripeMaxS, best_slots = 1 << 30;
  for (int s = kStripeMaxS; s >= 3; --s) {
    const int slots = ((nrb + s - 1) / s) * s;
    if (slots < best_slots) {
      best_slots = slots;
      best = s;
    }
  }
  return best;
}

// 16-byte vectors a lane loads per stripe (the stretch of S windows plus the
// segment phase, up to E-1 elements).
__host__ __device__ constexpr int stripe_nv(int ES, int S) { return (16 / ES - 1 + 4 * S + 16 / ES - 1) / (16 / ES); }

// Cut-out sizes of the map.  An even cut-out (the paper-window mode only,
// flags bits 3 and 4 for Ks and Kt) is mapped as the odd cut-out one pixel
// smaller: Eqs. 4-8 with even n_s read the pixels s < n_s - 1 and write the
// positions s' < n_s - 1, as the transpose of that cropped cut-out would
// (under the loop ranges' window); the last row or column stays zero.
__host__ __device__ inline int map_ks(const TileDesc& td) { return td.Ks - ((td.flags >> 3) & 1); }
__host__ __device__ inline int map_kt(const TileDesc& td) { return td.Kt - ((td.flags >> 4) & 1); }
// Source pixels of a tile's columns v0 .. v0+ncols-1: those with v < Ktm.
__host__ __device__ inline int tile_nseg(const TileDesc& td) {
  const int n = map_kt(td) - (int)td.v0;
  return n < 0 ? 0 : (n > (int)td.ncols ? (int)td.ncols : n);
}

// Row pitch (elements) of a tile whose slots have pitch P.
__host__ __device__ inline int row_pitch(int Ny, int P, int es) {
  const int sh = es == 4 ? 2 : 3;  // log2(16 / es)
  return ((Ny * P + (1 << sh) - 1) >> sh) << sh;
}

// ------------------------------------------------------------ host planning --
// Shared-memory bank wavefronts of the gather for one slot pitch P, averaged
// over pseudo-random segment phases and positions (they depend on buffer
// addresses unknown at planning time).  Mirrors the consumer's lane mapping:
// lane l of a warp step takes the chunk of elements e0 + l*EPL .. of one row.
inline double pitch_cost(int Ny, int Ks, int Kt, int ncols, int es, int P) {
  const int epl = 16 / es, E = 16 / es;
  (void)Ks;
  (void)Kt;
  uint32_t rng = 0x9e3779b9u ^ (uint32_t)((uint32_t)P * 2654435761u);
  long long total = 0;
  int count = 0;
  for (int trial = 0; trial < 48; ++trial) {
    rng = rng * 1664525u + 1013904223u;
    const int b0 = (int)((rng >> 8) % (uint32_t)Ny);
    rng = rng * 1664525u + 1013904223u;
    const int R = (int)((rng >> 8) % 64u) * E + (int)((rng >> 20) % (uint32_t)E);
    rng = rng * 1664525u + 1013904223u;
    const int e0 = (int)((rng >> 8) % (uint32_t)lfbp_max(1, ncols - 32 * epl));
    for (int sub = 0; sub < epl; ++sub) {
      long long words[32];
      int n = 0;
      for (int l = 0; l < 32; ++l) {
        const int vl = e0 + l * epl + sub;
        if (vl >= ncols) continue;
        const int b = (b0 + vl) % Ny;
        const long long idx = (long long)R + (long long)b * P + ncols - 1 - vl;
        words[n++] = (idx * es) / 4;
      }
      int worst = 0;
      for (int bank = 0; bank < 32; ++bank) {
        long long seen[32];
        int ns = 0;
        for (int i = 0; i < n; ++i) {
          if ((int)(words[i] % 32) != bank) continue;
          bool dup = false;
          for (int s = 0; s < ns; ++s) dup = dup || seen[s] == words[i];
          if (!dup) seen[ns++] = words[i];
        }
        worst = lfbp_max(worst, ns);
      }
      total += worst;
      ++count;
    }
  }
  return count ? (double)total / count : 0.0;
}

// The same for the stripe path (lfbp_stripes.cuh): lane 4s + g of a warp
// loads NV consecutive 16-byte vectors of segment (B + 4s + g) mod Ny from
// stage element R + ncols - 1 + b*P - V - 4s - g on (rounded down to 16
// bytes); each quarter-warp of a 16-byte load is one wavefront per distinct
// vector that shares a bank group with another.
inline double pitch_cost_stripes(int Ny, int ncols, int es, int P) {
  const int E = 16 / es;
  const int NV = stripe_nv(es, stripe_S((Ny + 3) >> 2));
  uint32_t rng = 0x85ebca6bu ^ (uint32_t)((uint32_t)P * 2246822519u);
  long long total = 0;
  int count = 0;
  for (int trial = 0; trial < 48; ++trial) {
    rng = rng * 1664525u + 1013904223u;
    const int B0 = (int)((rng >> 8) % (uint32_t)Ny);
    rng = rng * 1664525u + 1013904223u;
    const int R = (int)((rng >> 8) % (uint32_t)E);
    rng = rng * 1664525u + 1013904223u;
    const int V0 = (int)((rng >> 8) % (uint32_t)lfbp_max(1, ncols));
    long long unit[32];
    for (int l = 0; l < 32; ++l) {
      const int gs = l >> 2, g = l & 3;
      const int b = (B0 + 4 * gs + g) % Ny;
      const long long X = (long long)R + ncols - 1 + (long long)b * P - (V0 + 4 * gs) - g;
      const long long A = X >= 0 ? X / E : -((-X + E - 1) / E);  // floor(X / E)
      unit[l] = A;
    }
    for (int v = 0; v < NV; ++v) {
      for (int h = 0; h < 4; ++h) {
        int worst = 0;
        for (int bank = 0; bank < 8; ++bank) {
          long long seen[8];
          int ns = 0;
          for (int l = 8 * h; l < 8 * h + 8; ++l) {
            const long long u = unit[l] + v;
            if ((int)(((u % 8) + 8) % 8) != bank) continue;
            bool dup = false;
            for (int s2 = 0; s2 < ns; ++s2) dup = dup || seen[s2] == u;
            if (!dup) seen[ns++] = u;
          }
          worst = lfbp_max(worst, ns);
        }
        total += worst;
      }
      ++count;
    }
  }
  return count ? (double)total / count : 0.0;
}

// Tiles taken by the stripe consumer (lfbp_stripes.cuh) in either map mode.
__host__ __device__ inline bool stripe_shape(int Ny, int Ks, int Kt, int ncols, int es) {
  return LFBP_STRIPES && es == 2 && (((long long)Ks * Kt) & 3) == 1 && Ny >= 3 && ncols >= 8;
}

// Slot pitch for segments of ncols elements: P >= ncols + 2E - 2 (room for a
// copy widened to 16-byte boundaries), P = Ks*Kt (mod E), fewest conflicts.
inline int choose_pitch(int Ny, int Ks, int Kt, int ncols, int es) {
  const int E = 16 / es;
  const bool stripes = stripe_shape(Ny, Ks, Kt, ncols, es);
  const int KKm = (int)(((long long)Ks * Kt) % E);
  int P0 = ncols + 2 * E - 2;
  P0 += ((KKm - P0) % E + E) % E;
  int best = P0;
  double best_cost = 1e30;
  for (int x = 0; x < 8; ++x) {
    const int P = P0 + x * E;
    const double cost =
        stripes ? pitch_cost_stripes(Ny, ncols, es, P) : pitch_cost(Ny, Ks, Kt, ncols, es, P);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = P;
    }
  }
  return best;
}

// Tiling of one depth: rows per tile J, columns per tile V (V = Kt unless one
// row does not fit the target), counts of u- and v-blocks, and slot pitch.
struct DepthTiling {
  int J, V, nU, nV, P, RP;
  int max_tile_bytes;
};

inline DepthTiling tile_depth(int Ny, int Ks, int Kt, int es, int target) {
  DepthTiling d;
  const int E = 16 / es;
  int P = choose_pitch(Ny, Ks, Kt, Kt, es);
  const int row = row_pitch(Ny, P, es) * es;
  if (row <= target) {
    d.V = Kt;
    d.nV = 1;
    const int J = lfbp_max(1, lfbp_min(lfbp_min(Ks, kMaxTileRows), target / row));
    d.nU = (Ks + J - 1) / J;
    d.J = (Ks + d.nU - 1) / d.nU;
  } else {
    d.J = 1;
    d.nU = Ks;
    int nV = (row + target - 1) / target;
    for (;; ++nV) {
      const int V = (Kt + nV - 1) / nV;
      const int Pmax = V + 2 * E - 2 + 8 * E;  // largest pitch choose_pitch can return
      if (row_pitch(Ny, Pmax, es) * es <= target || V == 1) break;
    }
    d.V = (Kt + nV - 1) / nV;
    d.nV = (Kt + d.V - 1) / d.V;
    P = choose_pitch(Ny, Ks, Kt, d.V, es);
  }
  d.P = P;
  d.RP = row_pitch(Ny, P, es);
  d.max_tile_bytes = d.J * d.RP * es;
  return d;
}

// ---------------------------------------------------------------- PTX ----
// Under LFBP_HOST_EMULATION the including translation unit supplies host
// stand-ins for these primitives (and for the global-store helper and the
// shared-memory index check below), so that the tile code of this header can
// be run on the CPU with every memory access checked.
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
// 16-byte copy from global to shared memory through the load/store path
// (not the TMA unit); both addresses 16-byte aligned.  Completion is tracked
// per thread: cp_async_arrive_noinc makes an mbarrier arrival once all of the
// thread's earlier such copies have landed (the barrier's count includes it).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
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

template <class T>
__device__ __forceinline__ void st_global(T* p, T v) {
  *p = v;
}
template <class T>
__device__ __forceinline__ T lds(uint32_t addr);
template <>
__device__ __forceinline__ uint32_t lds<uint32_t>(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
template <>
__device__ __forceinline__ uint16_t lds<uint16_t>(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t addr) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}
// shared-memory load at a compile-time byte offset from a 32-bit address
template <class T, int OFF>
__device__ __forceinline__ T lds_off(uint32_t addr) {
  if constexpr (sizeof(T) == 4) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
    return v;
  } else {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1+%2];" : "=h"(v) : "r"(addr), "n"(OFF));
    return v;
  }
}
#define LFBP_SMEM_CHECK(idx)
#endif  // LFBP_HOST_EMULATION

// Self-checking build (LFBP_CHECK): every shared-memory load, global store and
// bulk copy of the tile code is checked against its buffer; the first
// violation is recorded in g_check (read by lfbp_sync_status) and the access
// is skipped.  No trap, no fault: a bad index costs a wrong value, not the GPU.
#if defined(LFBP_CHECK) && !defined(LFBP_HOST_EMULATION)
struct CheckWord {
  int code;  // 1 smem load, 2 global store, 3 bulk copy, 4 tail load
  int thread;
  int block;
  int pad;
  long long a, b;
};
static __device__ CheckWord g_check;
__device__ __forceinline__ void check_fail(int code, long long a, long long b) {
  if (atomicCAS(&g_check.code, 0, code) == 0) {
    g_check.thread = threadIdx.x;
    g_check.block = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    g_check.a = a;
    g_check.b = b;
  }
}
#define LFBP_CHECKED 1
#else
#define LFBP_CHECKED 0
#endif

// f(std::integral_constant<int, I>) for I = B .. E-1, unrolled at compile time
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

__device__ __forceinline__ int pos_mod(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// Producer side: the bulk copies of the tile's input segments into the stage.
// Shared by all 32 lanes of each of `np` warps; lane i of warp pw
// (0 <= pw < np) takes slots pw*32 + i, pw*32 + i + 32*np, ... (slot = j*Ny + b).
// A warp's bulk copies are accepted one lane at a time, so the copies of a
// tile with many short segments can be spread over several warps.
// tile_copies(..., count_only = true) returns the bytes this lane's copies
// bring in (for the barrier's expected transaction count) without issuing
// them; with count_only = false it issues them.  The last <16 bytes of an
// array that a 16-byte-widened copy would over-read are copied with ordinary
// loads instead.
__device__ __forceinline__ uint32_t tile_copies(const TileDesc& td, const unsigned char* in_depth,
                                                const unsigned char* in_safe_end,
                                                unsigned char* stage, uint32_t bar, int lane,
                                                int pw, int np, bool count_only) {
  const int es = (td.flags & 1) ? 2 : 4, E = 16 / es;
  const int Nx = td.Nx, Ny = td.Ny, Ks = td.Ks, Kt = td.Kt, P = td.P;
  const int RP = row_pitch(Ny, P, es);
  const int nslots = td.nrows * Ny;
  const int Ksm = map_ks(td), nseg = tile_nseg(td);
  const int cs = (Ksm - 1) / 2;
  const int t_lo = map_kt(td) - td.v0 - nseg;
  const uint32_t seg_bytes = (uint32_t)nseg * es;
  const unsigned long long KK = (unsigned long long)Ks * Kt;
  const unsigned long long NKK = (unsigned long long)Ny * KK;
  const FastDiv fNy = make_fastdiv(Ny), fNx = make_fastdiv(Nx);
  const int a0 = pos_mod(td.p + td.u0 - cs, Nx);
  const uintptr_t in_el = (uintptr_t)in_depth / es;
#if LFBP_CHECKED
  const int nrows_bytes = td.nrows * RP * es;
  const unsigned char* in_array = in_depth - td.off_bytes;
#endif
  // slot i = (row j, segment b): row j reads H[a_j][b][s_j][t_lo..], with
  // a_j = (p + u0 + j - c_s) mod Nx and s_j = Ksm - 1 - u0 - j (no copy for
  // the zero row of an even cut-out, s_j < 0, nor for an empty segment)
  const int slot0 = pw * 32 + lane, slot_step = 32 * np;
  const int jmax = (int)td.nrows < Ksm - (int)td.u0 ? (int)td.nrows : Ksm - (int)td.u0;  // rows with a source
  const int ncopy = nseg > 0 && jmax > 0 ? jmax * Ny : 0;
  (void)nslots;
  uint32_t my_bytes = 0;
  if (count_only) {
    for (int i = slot0; i < ncopy; i += slot_step) {
      const int j = (int)fdiv((uint32_t)i, fNy), b = i - j * Ny;
      const int a = (int)fmod_((uint32_t)(a0 + j), fNx);
      const unsigned long long seg =
          (unsigned long long)a * NKK + (unsigned long long)b * KK +
          (unsigned long long)(Ksm - 1 - td.u0 - j) * Kt + t_lo;
      const uintptr_t src = (uintptr_t)(in_depth + seg * es);
      const uintptr_t lo = src & ~(uintptr_t)15;
      uintptr_t hi = (src + seg_bytes + 15) & ~(uintptr_t)15;
      if (hi > (uintptr_t)in_safe_end) hi = (uintptr_t)in_safe_end;
      if (hi > lo) my_bytes += (uint32_t)(hi - lo);
    }
    return my_bytes;
  }
  bool fixed = false;
  for (int i = slot0; i < ncopy; i += slot_step) {
    const int j = (int)fdiv((uint32_t)i, fNy), b = i - j * Ny;
    const int a = (int)fmod_((uint32_t)(a0 + j), fNx);
    const unsigned long long seg0 =
        (unsigned long long)a * NKK + (unsigned long long)(Ksm - 1 - td.u0 - j) * Kt + t_lo;
    const unsigned long long seg = seg0 + (unsigned long long)b * KK;
    const uintptr_t src = (uintptr_t)(in_depth + seg * es);
    // phases (elements mod E) of segments (j, 0) and (j, b)
    const int ph0 = (int)((in_el + seg0) & (E - 1));
    const int phb = (int)((in_el + seg) & (E - 1));
    const int dst_el = j * RP + ph0 + b * P - phb;  // a multiple of E by the choice of P
    unsigned char* dst = stage + (size_t)dst_el * es;
    const uintptr_t lo = src & ~(uintptr_t)15;
    const uintptr_t end = src + seg_bytes;
    uintptr_t hi = (end + 15) & ~(uintptr_t)15;
    if (hi > (uintptr_t)in_safe_end) {
      hi = (uintptr_t)in_safe_end > lo ? (uintptr_t)in_safe_end : lo;
      // tail beyond the last full 16-byte block of the array: plain loads
      for (uintptr_t x = hi > src ? hi : src; x < end; x += es) {
#if LFBP_CHECKED
        if ((long long)(dst - stage) + (long long)(x - lo) + es > (long long)nrows_bytes ||
            x < (uintptr_t)in_array || x + es > (uintptr_t)in_safe_end + 16) {
          check_fail(4, (long long)(dst - stage) + (long long)(x - lo), (long long)nrows_bytes);
          continue;
        }
#endif
        if (es == 4)
          *(uint32_t*)(dst + (x - lo)) = __ldg((const unsigned int*)x);
        else
          *(uint16_t*)(dst + (x - lo)) = __ldg((const unsigned short*)x);
      }
      fixed = true;
    }
#if LFBP_CHECKED
    if (hi > lo && (dst < stage || (long long)(dst - stage) + (long long)(hi - lo) > (long long)nrows_bytes ||
                    ((uintptr_t)dst & 15) || (lo & 15) || ((hi - lo) & 15) ||
                    lo < (uintptr_t)in_array || hi > (uintptr_t)in_safe_end)) {
      check_fail(3, (long long)(dst - stage), (long long)(hi - lo));
      continue;
    }
#endif
    if (hi > lo) bulk_g2s(smem_addr(dst), (const void*)lo, (uint32_t)(hi - lo), bar);
  }
  if (fixed) fence_proxy_async_smem();
  return 0;
}

// Producer side through the load/store path: the same segments, widened to
// the same 16-byte boundaries and placed at the same stage addresses as
// tile_copies, moved as 16-byte cp.async copies.  Warp pw of np takes slots
// pw, pw + np, ... (slot = j*Ny + b); its lanes take the slot's 16-byte pieces.
// Used where the TMA unit's per-copy cost would bound the read rate, and for
// inputs in host memory.  The caller makes each lane arrive on the stage's
// barrier (cp_async_arrive_noinc) after this returns.
__device__ __forceinline__ void tile_copies_lsu(const TileDesc& td, const unsigned char* in_depth,
                                                const unsigned char* in_safe_end,
                                                unsigned char* stage, int lane, int pw, int np) {
  const int es = (td.flags & 1) ? 2 : 4, E = 16 / es;
  const int Nx = td.Nx, Ny = td.Ny, Ks = td.Ks, Kt = td.Kt, P = td.P;
  const int RP = row_pitch(Ny, P, es);
  const int Ksm = map_ks(td), nseg = tile_nseg(td);
  const int cs = (Ksm - 1) / 2;
  const int t_lo = map_kt(td) - td.v0 - nseg;
  const uint32_t seg_bytes = (uint32_t)nseg * es;
  const unsigned long long KK = (unsigned long long)Ks * Kt;
  const unsigned long long NKK = (unsigned long long)Ny * KK;
  const int a0 = pos_mod(td.p + td.u0 - cs, Nx);
  const uintptr_t in_el = (uintptr_t)in_depth / es;
#if LFBP_CHECKED
  const int nrows_bytes = td.nrows * RP * es;
  const unsigned char* in_array = in_depth - td.off_bytes;
#endif
  const int jmax = (int)td.nrows < Ksm - (int)td.u0 ? (int)td.nrows : Ksm - (int)td.u0;
  if (nseg <= 0 || jmax <= 0) return;
  const uint32_t stage_s = smem_addr(stage);
  // slots in (j, b) order, warp pw starting at slot pw; (j, b, a) advanced
  // incrementally by np slots per step
  int j = 0, b = pw;
  while (b >= Ny) { b -= Ny; ++j; }
  int a = a0 + j;
  while (a >= Nx) a -= Nx;
  for (; j < jmax;) {
    const unsigned long long seg0 =
        (unsigned long long)a * NKK + (unsigned long long)(Ksm - 1 - td.u0 - j) * Kt + t_lo;
    const unsigned long long seg = seg0 + (unsigned long long)b * KK;
    const uintptr_t src = (uintptr_t)(in_depth + seg * es);
    const int ph0 = (int)((in_el + seg0) & (E - 1));
    const int phb = (int)((in_el + seg) & (E - 1));
    const int dst_el = j * RP + ph0 + b * P - phb;  // a multiple of E by the choice of P
    const uintptr_t lo = src & ~(uintptr_t)15;
    const uintptr_t end = src + seg_bytes;
    uintptr_t hi = (end + 15) & ~(uintptr_t)15;
    if (hi > (uintptr_t)in_safe_end) {
      hi = (uintptr_t)in_safe_end > lo ? (uintptr_t)in_safe_end : lo;
      // tail beyond the last full 16-byte block of the array: plain loads, one
      // element per lane
      const uintptr_t x0 = hi > src ? hi : src;
      const uintptr_t x = x0 + (uintptr_t)lane * es;
      if (x < end) {
        unsigned char* d = stage + (size_t)dst_el * es + (x - lo);
#if LFBP_CHECKED
        if ((long long)(d - stage) + es > (long long)nrows_bytes || x < (uintptr_t)in_array ||
            x + es > (uintptr_t)in_safe_end + 16)
          check_fail(4, (long long)(d - stage), (long long)nrows_bytes);
        else
#endif
        if (es == 4)
          *(uint32_t*)d = __ldg((const unsigned int*)x);
        else
          *(uint16_t*)d = __ldg((const unsigned short*)x);
      }
    }
    const int npieces = hi > lo ? (int)((hi - lo) >> 4) : 0;
#if LFBP_CHECKED
    if (npieces && (dst_el * es < 0 || dst_el * es + npieces * 16 > nrows_bytes || ((dst_el * es) & 15) ||
                    lo < (uintptr_t)in_array || hi > (uintptr_t)in_safe_end)) {
      check_fail(3, (long long)dst_el * es, (long long)npieces * 16);
    } else
#endif
    for (int k = lane; k < npieces; k += 32)
      cp_async16(stage_s + (uint32_t)(dst_el * es + 16 * k), (const void*)(lo + 16 * (uintptr_t)k));
    // next slot of this warp
    b += np;
    while (b >= Ny) {
      b -= Ny;
      ++j;
      if (++a == Nx) a = 0;
    }
  }
}

#ifndef LFBP_HOST_EMULATION
// One warp's share of the tile's copies: the bytes of all its lanes are
// registered on `bar` with one expect_tx, then the copies are issued.  The
// caller arrives on `bar` afterwards (once per warp).
__device__ __forceinline__ void issue_tile_loads(const TileDesc& td, const unsigned char* in_depth,
                                                 const unsigned char* in_safe_end,
                                                 unsigned char* stage, uint32_t bar, int lane,
                                                 int pw, int np) {
  const uint32_t mine = tile_copies(td, in_depth, in_safe_end, stage, bar, lane, pw, np, true);
  const uint32_t total = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0 && total) mbar_expect_tx(bar, total);
  __syncwarp();
  tile_copies(td, in_depth, in_safe_end, stage, bar, lane, pw, np, false);
}
#endif

// Tile constants that depend only on the depth's sizes, the dtype, the mode
// and the tile's row and column counts (and, for an even cut-out, on whether
// the tile holds the zero column): computed on the host once per depth and
// tile shape (make_shape), stored in a table beside the work list, and copied
// into the tile context by one warp with coalesced loads.  All the divisions
// of the context are here.
struct alignas(16) TileShape {
  int Nx, Ny, Ks, Kt, ncols, nrows, L, P, RP, tile_bytes;
  int Ksm, Ktm;  // cut-out sizes of the map (Ks, Kt, or one less when even)
  int nseg;      // source pixels per segment: the columns v < Ktm of the tile
  int even;      // nonzero: an even cut-out (zero row / column, clamped reads)
  int Ks1, Kt1;  // Ks - 1, Kt - 1
  int es, mode;
  int nkk;       // (Ny*Ks*Kt) mod E
  int ktm;       // Kt mod E
  int kks;       // (Ks*Kt) mod 128/es
  int sbn;       // (128/es) mod Ny
  int cmn;       // ncols mod Ny
  int ngc;       // work items per run (element-walk path)
  int items;
  int ngm;       // 128-byte lines per run (any alignment), at least 2
  int nunits;    // warp steps of the tile (chunk path): ceil(Ny * ngm / 4)
  int fast;      // 1: chunk path (mode 0 or 1, ncols >= 16/es, Ny >= 16/es)
  int inl;       // 1: a one-row tile stores the chunks cut by its runs' ends in the main
                 // loop, element by element; 0: in an edge pass after it (runs shorter
                 // than kInlineEndsBytes, where the main loop's element stores cost more)
  uint32_t run_stride;  // bytes between runs q and q+1 (Ks*Kt*es < 2^32)
  uint32_t PES;  // P * es
  uint32_t D;    // bytes between diagonal neighbours: (P - 1) * es
  uint32_t W;    // bytes of Ny slots: Ny * P * es
  int cbb_add;   // a multiple of Ny that is >= 128/es
  int ctm, csm;  // c_t mod Ny, c_s mod Nx (c from the map's cut-out)
  // pair path (lfbp_pairs.cuh)
  int pair;      // 1: pair path (mode 0, Ks*Kt = 1 mod 16/es, Ny >= 16/es, ncols > 16/es)
  int pnd;       // anti-diagonals per tile row
  int pnpr;      // pair slots per anti-diagonal: (Ny - 1) / 2
  int pnu;       // anti-diagonals per row on which one slot can hold a unit
  int punits;    // pair units of the tile: nrows * pnpr * pnu
  FastDiv fpnd, fpnpr, fpnu;
  // stripe path (lfbp_stripes.cuh)
  int stripe;    // 1: stripe path (mode 0 or 1, Ks*Kt = 1 mod 4, Ny >= 3, ncols >= 8)
  int S;         // run blocks of 4 runs per stripe
  int ns;        // stripes per row and band
  int rowns;     // nrows * ns
  int nitems_s;  // stripes of the tile: bands * nrows * ns
  int nsteps_s;  // warp steps: ceil(nitems_s / 8)
  FastDiv fncols, fNy, fNx, fngc, fngm;
  FastDiv fns, frowns, fnb;  // by ns, rowns, nrows + 1
};
static_assert(sizeof(TileShape) % 16 == 0, "TileShape layout");

// The shape constants of a tile (host; the host emulation calls it too).
// flags as in TileDesc; v0: the tile's first column (only whether the tile
// reaches the map's last column matters).
__host__ __device__ inline TileShape make_shape(int Nx, int Ny, int Ks, int Kt, int es, int flags,
                                                int P, int nrows, int ncols, int v0) {
  TileShape s;
  const int E = 16 / es, GE = 128 / es;
  const long long KK = (long long)Ks * Kt;
  s.Nx = Nx;
  s.Ny = Ny;
  s.Ks = Ks;
  s.Kt = Kt;
  s.ncols = ncols;
  s.nrows = nrows;
  s.L = nrows * ncols;
  s.P = P;
  s.RP = row_pitch(Ny, P, es);
  s.tile_bytes = nrows * s.RP * es;
  s.Ksm = Ks - ((flags >> 3) & 1);
  s.Ktm = Kt - ((flags >> 4) & 1);
  {
    const int n = s.Ktm - v0;
    s.nseg = n < 0 ? 0 : (n > ncols ? ncols : n);
  }
  s.even = (flags >> 3) & 3;
  s.Ks1 = Ks - 1;
  s.Kt1 = Kt - 1;
  s.es = es;
  s.mode = (flags >> 1) & 3;
  s.nkk = (int)(((long long)Ny * KK) & (E - 1));
  s.ktm = Kt & (E - 1);
  s.kks = (int)(KK & (GE - 1));
  s.sbn = GE % Ny;
  s.cmn = ncols % Ny;
  {
    const int ng = (s.L + 2 * GE - 2) / GE;  // groups per run, any alignment
    s.ngc = (ng + kGroupsPerItem - 1) / kGroupsPerItem;
    s.items = ((Ny + 3) >> 2) * s.ngc;
    s.ngm = ng < 2 ? 2 : ng;
    s.nunits = (Ny * s.ngm + 3) >> 2;
  }
  s.fast = s.mode <= 1 && ncols >= E && Ny >= E;
  s.inl = nrows == 1 && ncols * es >= kInlineEndsBytes;
  s.run_stride = (uint32_t)(KK * es);
  s.PES = (uint32_t)P * es;
  s.D = (uint32_t)(P - 1) * es;
  s.W = (uint32_t)Ny * P * es;
  s.cbb_add = ((GE + Ny - 1) / Ny) * Ny;
  s.ctm = ((s.Ktm - 1) / 2) % Ny;
  s.csm = ((s.Ksm - 1) / 2) % Nx;
  s.fncols = make_fastdiv(ncols);
  s.fNy = make_fastdiv(Ny);
  s.fNx = make_fastdiv(Nx);
  s.fngc = make_fastdiv(s.ngc);
  s.fngm = make_fastdiv(s.ngm);
  s.pair = 0;
  s.pnd = s.pnpr = s.pnu = s.punits = 0;
  s.fpnd = s.fpnpr = s.fpnu = make_fastdiv(1);
  if (kPairs && !(flags & 32) && s.mode == 0 && s.fast && (KK & (E - 1)) == 1 && (Ny & 1) &&
      ncols > E) {
    s.pnd = (Ny + ncols - 2) / E + 2;
    s.pnpr = (Ny - 1) / 2;
    s.pnu = (ncols - E) / E + 2;
    const long long units = (long long)nrows * s.pnpr * s.pnu;
    if (units < (1 << 24) && s.pnpr >= 2 && s.pnd >= 2) {
      s.pair = 1;
      s.punits = (int)units;
      s.fpnd = make_fastdiv(s.pnd);
      s.fpnpr = make_fastdiv(s.pnpr);
      s.fpnu = make_fastdiv(s.pnu);
    }
  }
  s.stripe = 0;
  s.S = s.ns = s.rowns = s.nitems_s = s.nsteps_s = 0;
  s.fns = s.frowns = make_fastdiv(1);
  s.fnb = make_fastdiv(nrows + 1);
  if (!s.pair && s.mode <= 1 && stripe_shape(Ny, Ks, Kt, ncols, es)) {
    const int nrb = (Ny + 3) >> 2;
    const int S = stripe_S(nrb);
    const int nbands = (nrb + S - 1) / S;
    const int ns = (ncols - 1 + 4 * (S - 1)) / 4 + 1;
    const long long items = (long long)nbands * nrows * ns;
    if (items < 65535 && (long long)nrows * ns < 65535) {
      s.stripe = 1;
      s.S = S;
      s.ns = ns;
      s.rowns = nrows * ns;
      s.nitems_s = (int)items;
      s.nsteps_s = (s.nitems_s + 7) >> 3;
      s.fns = make_fastdiv(ns);
      s.frowns = make_fastdiv(s.rowns);
    }
  }
  return s;
}

// Shape class `cls` of a depth's tiles under tiling d: (last row block) +
// 2 (last column block); the other blocks have d.J rows and d.V columns.
inline TileShape depth_shape(const DepthTiling& d, int Nx, int Ny, int Ks, int Kt, int es,
                             int flags, int cls) {
  const int last_row = cls & 1, last_col = cls >> 1;
  const int nrows = last_row ? Ks - (d.nU - 1) * d.J : lfbp_min(d.J, Ks);
  const int v0 = last_col ? (d.nV - 1) * d.V : 0;
  const int ncols = last_col ? Kt - v0 : lfbp_min(d.V, Kt);
  return make_shape(Nx, Ny, Ks, Kt, es, flags, d.P, nrows, ncols, v0);
}

// The context of one tile: its shape constants plus the fields that depend on
// the tile's position (p, u0, v0) and on the buffers.  Built once per tile in
// shared memory; every consumer thread copies it into registers before its
// gather loop (a copy in registers cannot be aliased by the gather's global
// stores, so it is not re-read after each store).
struct alignas(16) TileCtx : TileShape {
  uint32_t stage_s;         // shared-memory address of the stage
  uint32_t tab_s;           // shared-memory address of the row-base table: nrows + 1 ints
  unsigned char* out_run0;  // byte address of run q = 0 at (u0, v0)
  unsigned char* out_lo;    // the depth's output bytes [out_lo, out_hi)
  unsigned char* out_hi;
  int p, u0, v0;
  int cb;    // (v0 - c_t) mod Ny
  int cbb;   // cb + cbb_add
  int ap0;   // (p + u0 - c_s) mod Nx
  int s0;    // Ksm - 1 - u0
  int inm;   // phase (mod E) of the input depth base + t_lo, in elements
  int om0;   // absolute element index of run q = 0, mod 128/es
  int rb0;   // row base of row 0 (elements): R_0 + nseg - 1
  uint32_t A0;  // stage_s + rb0 * es
  // paper-window masks (modes 1 and 2), as per-tile bounds on row j, column
  // vl, run q and cells a, b (see keep_elem)
  int m1_j0, m1_jw, m1_q0, m2_a, m2_b, jlim, vlim;
};

// Row base of tile row j (elements): the stage index of the segment (j, 0)'s
// element for column 0, i.e. j*RP + R_j + nseg - 1 with R_j the 16-byte phase
// of that segment's first element; row j of segment b then holds output
// column vl at row_base(j) + b*P - vl.  Defined for j = nrows as well (the
// entry past the last row is read but never dereferenced).  inm, s0 and ap0 as
// in TileCtx.
__device__ __forceinline__ int row_base(const TileShape& s, int inm, int s0, int ap0, int j) {
  const int E = 16 / s.es;
  const int a = (int)fmod_((uint32_t)(ap0 + j), s.fNx);
  return j * s.RP + ((inm + a * s.nkk + (s0 - j) * s.ktm) & (E - 1)) + s.nseg - 1;
}

// The shape part of the context: lane `lane` of a full warp copies words
// lane, lane + 32, ... of the shape record (coalesced loads).
__device__ __forceinline__ void copy_shape(TileCtx& c, const TileShape* shp, int lane) {
  constexpr int kWords = (int)(sizeof(TileShape) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(shp);
  uint32_t* dst = reinterpret_cast<uint32_t*>(static_cast<TileShape*>(&c));
  for (int w = lane; w < kWords; w += 32) dst[w] = src[w];
}

// The tile part of the context, in four independent parts (part 0..3), each
// run by one thread, plus the row-base table (rows part, part + 4, ...).
// `shp` is the tile's shape record (it may be c itself once c holds it; the
// parts write only tile fields).
__device__ __forceinline__ void make_ctx_tile(TileCtx& c, const TileDesc& td, const TileShape* shp,
                                              const unsigned char* stage,
                                              const unsigned char* in_depth,
                                              unsigned char* out_depth, int* tab, int part) {
  const TileShape& s = *shp;
  const int ES = s.es, E = 16 / ES, GE = 128 / ES;
  const int p = td.p, u0 = td.u0, v0 = td.v0;
  // values every part needs
  const int s0 = s.Ksm - 1 - u0;
  const int ap0 = (int)fmod_((uint32_t)(p + u0 + s.Nx - s.csm), s.fNx);
  const int t_lo = s.Ktm - v0 - s.nseg;
  const int inm = (int)((((uintptr_t)in_depth / ES) + (unsigned long long)t_lo) & (E - 1));
  for (int j = part; j <= s.nrows; j += 4) tab[j] = row_base(s, inm, s0, ap0, j);
  switch (part) {
    case 0:
      c.stage_s = smem_addr(stage);
      c.tab_s = smem_addr(tab);
      c.p = p;
      c.u0 = u0;
      c.v0 = v0;
      c.s0 = s0;
      c.ap0 = ap0;
      c.inm = inm;
      break;
    case 1: {
      const int cb = (int)fmod_((uint32_t)(v0 + s.Ny - s.ctm), s.fNy);
      c.cb = cb;
      c.cbb = cb + s.cbb_add;
      c.rb0 = row_base(s, inm, s0, ap0, 0);
      c.A0 = smem_addr(stage) + (uint32_t)c.rb0 * ES;
      break;
    }
    case 2: {
      const unsigned long long run0 =
          ((unsigned long long)p * s.Ny * s.Ks + u0) * s.Kt + v0;  // elements
      c.out_run0 = out_depth + run0 * ES;
      c.om0 = (int)((((uintptr_t)c.out_run0) / ES) & (GE - 1));
      c.out_lo = out_depth;
      c.out_hi = out_depth + (unsigned long long)s.Nx * s.Ny * s.Ks * s.Kt * ES;
      break;
    }
    case 3:
      if (s.mode != 0) {
        const int hx = (s.Nx - 1) >> 1, hy = (s.Ny - 1) >> 1;
        c.jlim = s.Ksm - u0;
        c.vlim = s.Ktm - v0;
        const int j0 = hx - p - u0;
        const int j1 = lfbp_dmin(s.Ks - 1 + j0, c.jlim - 1);
        c.m1_j0 = j1 >= j0 ? j0 : (1 << 20);  // no row kept: an empty range
        c.m1_jw = j1 >= j0 ? j1 - j0 : 0;
        c.m1_q0 = hy - v0;
        c.m2_a = s0 - hx;
        c.m2_b = s.Ktm - 1 - v0 - hy;
      }
      break;
    default:
      break;
  }
}

// The whole context from one thread (used where no warp is at hand).
__device__ __forceinline__ void make_ctx(TileCtx& c, const TileDesc& td, const TileShape* shp,
                                         const unsigned char* stage, const unsigned char* in_depth,
                                         unsigned char* out_depth, int* tab) {
  for (int l = 0; l < 32; ++l) copy_shape(c, shp, l);
  for (int part = 0; part < 4; ++part)
    make_ctx_tile(c, td, shp, stage, in_depth, out_depth, tab, part);
}

template <class T>
__device__ __forceinline__ T smem_load(const TileCtx& c, int idx) {
#if LFBP_CHECKED
  if (idx < 0 || (long long)(idx + 1) * (long long)sizeof(T) > c.tile_bytes) {
    check_fail(1, idx, c.tile_bytes);
    return (T)0;
  }
#endif
  return lds<T>(c.stage_s + (uint32_t)idx * (uint32_t)sizeof(T));
}

template <class T, int OFF>
__device__ __forceinline__ T smem_load_off(const TileCtx& c, uint32_t addr) {
#if LFBP_CHECKED
  const long long rel = (long long)addr + OFF - (long long)c.stage_s;
  if (rel < 0 || rel + (long long)sizeof(T) > c.tile_bytes) {
    check_fail(1, rel, c.tile_bytes);
    return (T)0;
  }
#endif
  (void)c;
  return lds_off<T, OFF>(addr);
}

__device__ __forceinline__ uint4 pack16(const uint32_t (&v)[4]) {
  uint4 w;
  w.x = v[0];
  w.y = v[1];
  w.z = v[2];
  w.w = v[3];
  return w;
}
__device__ __forceinline__ uint4 pack16(const uint16_t (&v)[8]) {
  uint4 w;
  w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
  w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
  w.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
  w.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
  return w;
}

__device__ __forceinline__ void store_out16(const TileCtx& c, unsigned char* p, uint4 v) {
#if LFBP_CHECKED
  if (p < c.out_lo || p + 16 > c.out_hi || ((uintptr_t)p & 15)) {
    check_fail(2, (long long)(p - c.out_lo), (long long)(c.out_hi - c.out_lo));
    return;
  }
#endif
  (void)c;
  st_global(reinterpret_cast<uint4*>(p), v);
}

__device__ __forceinline__ void store_out8(const TileCtx& c, unsigned char* p, uint32_t lo,
                                           uint32_t hi) {
#if LFBP_CHECKED
  if (p < c.out_lo || p + 8 > c.out_hi || ((uintptr_t)p & 7)) {
    check_fail(2, (long long)(p - c.out_lo), (long long)(c.out_hi - c.out_lo));
    return;
  }
#endif
  (void)c;
  uint2 v;
  v.x = lo;
  v.y = hi;
  st_global(reinterpret_cast<uint2*>(p), v);
}

// 16-byte shared-memory load of the tile's stage at a 16-byte-aligned address.
__device__ __forceinline__ uint4 lds_v4(const TileCtx& c, uint32_t addr) {
#if LFBP_CHECKED
  const long long rel = (long long)addr - (long long)c.stage_s;
  if (rel < 0 || rel + 16 > c.tile_bytes || (rel & 15)) {
    check_fail(1, rel, c.tile_bytes);
    return make_uint4(0, 0, 0, 0);
  }
#endif
  (void)c;
  return lds128(addr);
}

template <class T>
__device__ __forceinline__ void store_out(const TileCtx& c, T* p, T v) {
#if LFBP_CHECKED
  const unsigned char* b = reinterpret_cast<const unsigned char*>(p);
  if (b < c.out_lo || b + sizeof(T) > c.out_hi || ((uintptr_t)b & (sizeof(T) - 1))) {
    check_fail(2, (long long)(b - c.out_lo), (long long)(c.out_hi - c.out_lo));
    return;
  }
#endif
  (void)c;
  st_global(p, v);
}

// Shared-memory element index of run-element e of run q, computed from
// scratch; also returns row j, column vl, source b and cell a (for masks).
template <int ES>
__device__ __forceinline__ int src_index(const TileCtx& c, int q, int e, int& j, int& vl, int& b,
                                         int& a) {
  constexpr int E = 16 / ES;
  j = (int)fdiv((uint32_t)e, c.fncols);
  vl = e - j * c.ncols;
  a = (int)fmod_((uint32_t)(c.ap0 + j), c.fNx);
  const int ph = (c.inm + a * c.nkk + (c.s0 - j) * c.ktm) & (E - 1);
  b = (int)fmod_((uint32_t)(q + c.cb + vl), c.fNy);
  return j * c.RP + ph + b * c.P + c.nseg - 1 - vl;
}

template <int MODE>
__device__ __forceinline__ bool keep_elem(const TileCtx& c, int q, int j, int vl, int b, int a) {
  if (MODE == 0) return true;
  // rows and columns past the map's cut-out (the last of an even one) are zero
  if (MODE == 1) {
    // forward paper window, on the output position (p, u, q, v):
    // p + u0 + j - h_x in [0, Ks-1], u0 + j < Ksm, q + v0 + vl - h_y in [0, Kt-1], v0 + vl < Ktm
    return (unsigned)(j - c.m1_j0) <= (unsigned)c.m1_jw &&
           (unsigned)(q + vl - c.m1_q0) <= (unsigned)c.Kt1 && vl < c.vlim;
  }
  // adjoint of the paper window, on the source position (a, s, b, t):
  // a + s - h_x in [0, Ks-1], b + t - h_y in [0, Kt-1], and the output inside the map's cut-out
  return j < c.jlim && vl < c.vlim && (unsigned)(a - j + c.m2_a) <= (unsigned)c.Ks1 &&
         (unsigned)(b - vl + c.m2_b) <= (unsigned)c.Kt1;
}

// n / d for d >= 2 (no special case for d = 1); exact while n*d < 2^32.
__device__ __forceinline__ uint32_t fdiv2(uint32_t n, FastDiv f) { return __umulhi(n, f.m); }
__device__ __forceinline__ uint32_t fmod2(uint32_t n, FastDiv f) { return n - fdiv2(n, f) * f.d; }

template <class T>
__device__ __forceinline__ T smem_load_at(const TileCtx& c, uint32_t addr) {
#if LFBP_CHECKED
  const long long rel = (long long)addr - (long long)c.stage_s;
  if (rel < 0 || rel + (long long)sizeof(T) > c.tile_bytes) {
    check_fail(1, rel, c.tile_bytes);
    return (T)0;
  }
#endif
  (void)c;
  return lds<T>(addr);
}

// Entry j (0 <= j <= nrows) of the tile's row-base table.
__device__ __forceinline__ int tab_load(const TileCtx& c, int j) {
#if LFBP_CHECKED
  if (j < 0 || j > c.nrows) {
    check_fail(5, j, c.nrows);
    return 0;
  }
#endif
  return (int)lds<uint32_t>(c.tab_s + 4u * (uint32_t)j);
}

// Consumer side, chunk path (transpose mode, ncols >= 16/es, Ny >= 16/es).
// The tile's Ny runs are cut into ngm aligned 128-byte lines each (lines past
// a run's end are skipped); warp step u covers lines 4u .. 4u+3 of the
// flattened (run, line) sequence, 8 lanes per line, one 16-byte chunk per
// lane.  Chunk element k of run element e + k sits in row j, column vl + k
// (or, past the row end, in row j+1), segment b + k mod Ny:
//     address = A + k*D - W*[k >= Ny - b]                 (same row)
//             = B + k*D - W*[k >= kx + Ny - bq0]          (next row, k >= kx)
// with D the diagonal stride, W the bytes of Ny slots, kx = ncols - vl and bq0
// the segment of column 0.  At most one wrap and one row crossing fall in a
// chunk because Ny and ncols are at least its element count.  Chunks cut by
// a run's ends store element by element.  `rot` rotates the step-to-warp
// assignment from tile to tile so that the warps share the remainder steps.
// MASK (the paper-window mode, Fig. 10's loop ranges): element k is kept
// iff its output position has p + u in [h_x, Ks - 1 + h_x] and q + v in
// [h_y, Kt - 1 + h_y]; the others are written as zero.
// Stage addresses of one chunk of the chunk path: chunk element 0 is run
// element e of run q.  A, kwA: address of element 0 and the first element that
// wraps from segment Ny-1 to 0 (same row); B, kwB: the same for the elements
// k >= kx of the next row (kx = EPL when the chunk stays in one row).
struct ChunkAddr {
  uint32_t A, B;
  int kwA, kx, kwB;
  int j, vl;  // row and column of chunk element 0 (used by the paper-window mask)
};

template <int ES, bool ONEROW>
__device__ __forceinline__ ChunkAddr chunk_addr(const TileCtx& c, int q, int e) {
  constexpr int EPL = 16 / ES;
  ChunkAddr s;
  const int Ny = c.Ny;
  s.kx = EPL;
  s.kwB = EPL;
  s.B = 0;
  if (ONEROW) {
    const int b = (int)fmod2((uint32_t)(q + c.cbb + e), c.fNy);
    s.A = c.A0 + (uint32_t)b * c.PES - (uint32_t)e * ES;
    s.kwA = Ny - b;
    s.j = 0;
    s.vl = e;
  } else {
    const int j = e > 0 ? (int)fdiv2((uint32_t)e, c.fncols) : 0;
    const int vl = e - j * c.ncols;
    const int rbj = tab_load(c, j);
    const int rbn = tab_load(c, j + 1);
    const int b = (int)fmod2((uint32_t)(q + c.cbb + vl), c.fNy);
    s.A = c.stage_s + (uint32_t)(rbj + b * c.P - vl) * ES;
    s.kwA = Ny - b;
    s.kx = c.ncols - vl;
    int bq0 = q + c.cb;
    if (bq0 >= Ny) bq0 -= Ny;
    s.B = c.stage_s + (uint32_t)(rbn + bq0 * c.P) * ES - (uint32_t)s.kx * c.D;
    s.kwB = s.kx + Ny - bq0;
    s.j = j;
    s.vl = vl;
  }
  return s;
}

// Paper-window mask of chunk element k (run q): rows j (k < kx) or j + 1,
// columns vl + k or k - kx; see gather_chunks.  EVEN: the tile is an even
// cut-out, whose last column (vl >= vlim) is zero as well.
template <bool ONEROW, bool EVEN>
__device__ __forceinline__ bool chunk_keep(const TileCtx& c, const ChunkAddr& s, int q, int k) {
  const bool nxt = !ONEROW && k >= s.kx;
  const int j = nxt ? s.j + 1 : s.j;
  const int vl = nxt ? k - s.kx : s.vl + k;
  return (unsigned)(j - c.m1_j0) <= (unsigned)c.m1_jw &&
         (unsigned)(q + vl - c.m1_q0) <= (unsigned)c.Kt1 && (!EVEN || vl < c.vlim);
}

// The same test for all E elements of a chunk at once, as a bit mask (bit k:
// element k kept).  Along a chunk the row is j (k < kx) or j + 1, and the
// column tests of Eqs. 4-9's loop ranges keep a contiguous range of k in each
// row, so the mask is at most two bit ranges.
__device__ __forceinline__ uint32_t bit_range(int lo, int hi) {
  return lo > hi ? 0u : (2u << hi) - (1u << lo);  // bits lo..hi, 0 <= lo, hi < 31
}
template <bool ONEROW, bool EVEN, int E>
__device__ __forceinline__ uint32_t chunk_keep_mask(const TileCtx& c, const ChunkAddr& s, int q) {
  const int kx = ONEROW ? E : (s.kx < E ? s.kx : E);  // first element of row j + 1
  // row j: columns vl + k, kept for q + vl + k - m1_q0 in [0, Kt1] (and vl + k < vlim)
  uint32_t m = 0;
  if ((unsigned)(s.j - c.m1_j0) <= (unsigned)c.m1_jw) {
    int lo = c.m1_q0 - q - s.vl, hi = lo + c.Kt1;
    if (EVEN && c.vlim - 1 - s.vl < hi) hi = c.vlim - 1 - s.vl;
    lo = lo < 0 ? 0 : lo;
    hi = hi > kx - 1 ? kx - 1 : hi;
    m = bit_range(lo, hi);
  }
  // row j + 1: columns k - kx
  if (!ONEROW && kx < E && (unsigned)(s.j + 1 - c.m1_j0) <= (unsigned)c.m1_jw) {
    int lo = kx + c.m1_q0 - q, hi = lo + c.Kt1;
    if (EVEN && kx + c.vlim - 1 < hi) hi = kx + c.vlim - 1;
    lo = lo < kx ? kx : lo;
    hi = hi > E - 1 ? E - 1 : hi;
    m |= bit_range(lo, hi);
  }
  return m;
}

// MASK: 0 none (transpose mode), 1 the paper window on an odd cut-out, 2 the
// paper window on an even cut-out.
template <class T, int MASK, bool ONEROW>
__device__ __forceinline__ T masked(const TileCtx& c, const ChunkAddr& s, int q, int k, T x) {
  if (MASK && !chunk_keep<ONEROW, MASK == 2>(c, s, q, k)) return (T)0;
  return x;
}

// stage address of chunk element k
template <bool ONEROW>
__device__ __forceinline__ uint32_t chunk_elem(const TileCtx& c, const ChunkAddr& s, int k) {
  if (ONEROW) {
    uint32_t a = s.A + (uint32_t)k * c.D;
    if (k >= s.kwA) a -= c.W;
    return a;
  }
  const bool nxt = k >= s.kx;
  uint32_t a = (nxt ? s.B : s.A) + (uint32_t)k * c.D;
  if (k >= (nxt ? s.kwB : s.kwA)) a -= c.W;
  return a;
}

// The same, for a chunk whose elements may be masked: a masked element in
// the zero column of an even cut-out (MASK == 2) can sit one element before
// the stage; it is read inside the stage instead (the value is dropped
// either way).
template <int MASK, bool ONEROW>
__device__ __forceinline__ uint32_t chunk_elem_c(const TileCtx& c, const ChunkAddr& s, int k) {
  const uint32_t a = chunk_elem<ONEROW>(c, s, k);
  return MASK == 2 && (int)(a - c.stage_s) < 0 ? c.stage_s : a;
}

template <int ES, bool ONEROW, int MASK>
__device__ __forceinline__ void gather_chunks(const TileCtx& c, int w, int nwarps, int lane,
                                              int rot) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  constexpr int EPL = 16 / ES;  // elements per chunk
  constexpr int GE = 8 * EPL;   // elements per 128-byte line
  const int r = lane >> 3;
  const int lane_el = (lane & 7) * EPL;
  const int Ny = c.Ny, L = c.L;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  // Chunks cut by a run's end: one-row tiles with long runs (c.inl) store
  // them element by element in the step that meets them; other tiles leave
  // them to an edge pass after the loop (measured: each is the faster choice
  // for its kind of tile).
  const bool inl = ONEROW && c.inl;
  for (int u = first; u < c.nunits; u += nwarps) {
    const int f = u * 4 + r;
    const int q = (int)fdiv2((uint32_t)f, c.fngm);
    if (q >= Ny) continue;
    const int g = f - q * c.ngm;
    const int m = (c.om0 + q * c.kks) & (GE - 1);  // run q's first element within its line
    const int e = g * GE + lane_el - m;            // run element of chunk element 0
    const bool whole = e >= 0 && e + EPL <= L;
    if (inl ? (e >= L || e <= -EPL) : !whole) continue;
    unsigned char* dst =
        c.out_run0 + (unsigned long long)(uint32_t)q * c.run_stride + (long long)e * ES;
    const ChunkAddr s = chunk_addr<ES, ONEROW>(c, q, e);
    if (whole) {
      T v[EPL];
      const uint32_t keep = MASK ? chunk_keep_mask<ONEROW, MASK == 2, EPL>(c, s, q) : 0u;
      static_for<0, EPL>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const T x = smem_load_at<T>(c, chunk_elem_c<MASK, ONEROW>(c, s, k));
        v[k] = (!MASK || ((keep >> k) & 1u)) ? x : (T)0;
      });
      store_out16(c, dst, pack16(v));
    } else {
#pragma unroll
      for (int k = 0; k < EPL; ++k) {
        if (e + k < 0 || e + k >= L) continue;
        store_out(c, reinterpret_cast<T*>(dst) + k,
                  masked<T, MASK, ONEROW>(c, s, q, k, smem_load_at<T>(c, chunk_elem_c<MASK, ONEROW>(c, s, k))));
      }
    }
  }
  if (inl) return;
  // edge pass: the first and the last chunk of every run where a run end cuts
  // them, element by element; edge chunk i goes to the warp whose rotated
  // index is i mod nwarps, so each warp takes at most a few of them
  for (int i = first + nwarps * lane; i < 2 * Ny; i += 32 * nwarps) {
    const int q = i >> 1;
    const int m = (c.om0 + q * c.kks) & (GE - 1);
    const int e0 = -(m & (EPL - 1));  // start of the chunk holding run element 0
    int e = e0;
    if (i & 1) {
      e = e0 + (((L - 1 - e0) / EPL) * EPL);  // chunk holding the run's last element
      if (e + EPL <= L || e == e0) continue;   // whole, or the same chunk as the first
    } else if (e0 == 0 && EPL <= L) {
      continue;  // the first chunk is whole
    }
    unsigned char* dst =
        c.out_run0 + (unsigned long long)(uint32_t)q * c.run_stride + (long long)e * ES;
    const ChunkAddr s = chunk_addr<ES, ONEROW>(c, q, e);
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
      if (e + k < 0 || e + k >= L) continue;
      store_out(c, reinterpret_cast<T*>(dst) + k,
                masked<T, MASK, ONEROW>(c, s, q, k, smem_load_at<T>(c, chunk_elem_c<MASK, ONEROW>(c, s, k))));
    }
  }
}

// Consumer side, element-walk path (paper-window modes, and tiles whose rows
// or cells are shorter than a chunk): gather the tile from the stage through
// the index map and write its Ny output runs with 16-byte stores.  `w` is this warp's index
// among the `nwarps` consumer warps of the CTA; `rot` rotates the item-to-warp
// assignment from tile to tile so that the warps share the remainder items.
// Work item = 4 runs x kGroupsPerItem groups; a group is one 128-byte stretch
// of a run, 16 bytes per lane.  Inside a row, consecutive output elements walk
// the diagonal b -> b+1 (mod Ny), t -> t-1 of the stage: one IMAD per element
// for the address.  Every path keeps the walk's state (row j, cell a, column
// vl, segment b, row base) incrementally; only an item's start is computed
// with divisions.
template <int ES, int MODE>
__device__ __forceinline__ void gather_tile(const TileCtx& c, int w, int nwarps, int lane,
                                            int rot) {
  using T = typename std::conditional<ES == 4, uint32_t, uint16_t>::type;
  constexpr int E = 16 / ES;
  constexpr int EPL = 16 / ES;  // elements per lane and group (one 16-byte store)
  constexpr int GE = 8 * EPL;   // elements per run and group (128 bytes)
  const int r = lane >> 3, k = lane & 7;
  const int Ny = c.Ny, Nx = c.Nx, L = c.L, P = c.P, ncols = c.ncols, RP = c.RP;
  const uint32_t PES = (uint32_t)P * ES;
  int first = (w - rot) % nwarps;
  if (first < 0) first += nwarps;
  for (int it = first; it < c.items; it += nwarps) {
    const int qb = (int)fdiv((uint32_t)it, c.fngc);
    const int gc = it - qb * c.ngc;
    const int q = qb * 4 + r;
    if (q >= Ny) continue;
    const int m = (c.om0 + q * c.kks) & (GE - 1);
    unsigned char* orow = c.out_run0 + (long long)q * c.run_stride;
    int e = gc * (kGroupsPerItem * GE) + k * EPL - m;  // this lane's first element
    const int pos = e < 0 ? 0 : e;
    if (pos >= L) continue;
    // walk state at element `pos`
    int j, vl, b, a;
    int rb = src_index<ES>(c, q, pos, j, vl, b, a);  // = row base + b*P - vl
    rb += vl - b * P;                                 // row base: j*RP + phase_j + ncols - 1
    const int bq0 = (int)fmod_((uint32_t)(q + c.cb), c.fNy);  // segment of column 0
#pragma unroll 1
    for (int g = 0; g < kGroupsPerItem; ++g, e += GE) {
      if (e >= L) break;
      const int i0 = e < 0 ? -e : 0;  // first element of the group inside the run
      const bool allv = i0 == 0 && e + EPL <= L;
      T v[EPL];
      if (MODE == 0 && allv && vl + EPL <= ncols) {
        // whole group inside one row and inside the run
        const uint32_t X = c.stage_s + (uint32_t)(rb - vl - (EPL - 1)) * ES;
        int bb = b;
        static_for<0, EPL>([&](auto ic) {
          constexpr int ii = decltype(ic)::value;
          v[ii] = smem_load_off<T, (EPL - 1 - ii) * ES>(c, (uint32_t)bb * PES + X);
          bb = bb + 1 == Ny ? 0 : bb + 1;
        });
        store_out16(c, orow + (long long)e * ES, pack16(v));
      } else {
        // row crossings, run ends, masks: element by element, same walk
        int tv = vl, tb = b, tj = j, ta = a, trb = rb;
#pragma unroll
        for (int ii = 0; ii < EPL; ++ii) {
          v[ii] = 0;
          if (ii < i0 || e + ii >= L) continue;
          const int ix = trb + tb * P - tv;  // -1 only for a masked zero-column element
          T x = smem_load<T>(c, ix < 0 ? 0 : ix);
          if (!keep_elem<MODE>(c, q, tj, tv, tb, ta)) x = 0;
          v[ii] = x;
          if (!allv) store_out(c, reinterpret_cast<T*>(orow) + (e + ii), x);
          ++tv;
          tb = tb + 1 == Ny ? 0 : tb + 1;
          if (tv == ncols) {  // next row
            tv = 0;
            ++tj;
            ta = ta + 1 == Nx ? 0 : ta + 1;
            trb = tj * RP + ((c.inm + ta * c.nkk + (c.s0 - tj) * c.ktm) & (E - 1)) + c.nseg - 1;
            tb = bq0;
          }
        }
        if (allv) store_out16(c, orow + (long long)e * ES, pack16(v));
      }
      // move the walk to the next group's first element
      const int d = e < 0 ? e + GE : GE;
      vl += d;
      b += d == GE ? c.sbn : (int)fmod_((uint32_t)d, c.fNy);
      if (b >= Ny) b -= Ny;
      if (vl >= ncols) {
        do {
          vl -= ncols;
          ++j;
          a = a + 1 == Nx ? 0 : a + 1;
          b -= c.cmn;
          if (b < 0) b += Ny;
        } while (vl >= ncols);
        rb = j * RP + ((c.inm + a * c.nkk + (c.s0 - j) * c.ktm) & (E - 1)) + c.nseg - 1;
      }
    }
  }
}

}  // namespace lfbp

#include "lfbp_stripes.cuh"
#include "lfbp_pairs.cuh"

namespace lfbp {

// Consumer side, given the tile's context (in shared memory).
__device__ __forceinline__ void gather_tile_ctx(const TileCtx& cs, int w, int nwarps, int lane,
                                                int rot = 0) {
  if (cs.pair) {
    gather_pairs_ctx(cs, w, nwarps, lane, rot);
    return;
  }
#if !defined(LFBP_HOST_EMULATION) && LFBP_STRIPES
  if (cs.stripe) {
    gather_stripes_ctx(cs, w, nwarps, lane, rot);
    return;
  }
#endif
  const TileCtx c = cs;  // into registers, once per tile
  if (c.fast) {
    if (c.mode == 0) {
      if (c.es == 4) {
        if (c.nrows == 1)
          gather_chunks<4, true, 0>(c, w, nwarps, lane, rot);
        else
          gather_chunks<4, false, 0>(c, w, nwarps, lane, rot);
      } else {
        if (c.nrows == 1)
          gather_chunks<2, true, 0>(c, w, nwarps, lane, rot);
        else
          gather_chunks<2, false, 0>(c, w, nwarps, lane, rot);
      }
    } else if (!c.even) {
      if (c.es == 4) {
        if (c.nrows == 1)
          gather_chunks<4, true, 1>(c, w, nwarps, lane, rot);
        else
          gather_chunks<4, false, 1>(c, w, nwarps, lane, rot);
      } else {
        if (c.nrows == 1)
          gather_chunks<2, true, 1>(c, w, nwarps, lane, rot);
        else
          gather_chunks<2, false, 1>(c, w, nwarps, lane, rot);
      }
    } else {
      if (c.es == 4) {
        if (c.nrows == 1)
          gather_chunks<4, true, 2>(c, w, nwarps, lane, rot);
        else
          gather_chunks<4, false, 2>(c, w, nwarps, lane, rot);
      } else {
        if (c.nrows == 1)
          gather_chunks<2, true, 2>(c, w, nwarps, lane, rot);
        else
          gather_chunks<2, false, 2>(c, w, nwarps, lane, rot);
      }
    }
    return;
  }
  if (c.es == 4) {
    if (c.mode == 0)
      gather_tile<4, 0>(c, w, nwarps, lane, rot);
    else if (c.mode == 1)
      gather_tile<4, 1>(c, w, nwarps, lane, rot);
    else
      gather_tile<4, 2>(c, w, nwarps, lane, rot);
  } else {
    if (c.mode == 0)
      gather_tile<2, 0>(c, w, nwarps, lane, rot);
    else if (c.mode == 1)
      gather_tile<2, 1>(c, w, nwarps, lane, rot);
    else
      gather_tile<2, 2>(c, w, nwarps, lane, rot);
  }
}

}  // namespace lfbp
