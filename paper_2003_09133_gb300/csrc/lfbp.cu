// lfbp: H -> H' backprojection-array construction on one GPU (sm_103a).
//
// Kernels (see lfbp_device.cuh for the tile and the index map):
//   k_gather_depth       one tile per CTA, one launch per depth (the plain form)
//   k_gather_persistent  persistent CTAs over a ragged work list of all depths
//                        of all arrays; producer warps stream tiles into a
//                        ring of shared-memory stages with TMA bulk copies,
//                        consumer warps gather and store (the batched form)
// and the C-ABI of include/lfbp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "lfbp.h"
#include "lfbp_device.cuh"
#include "lfbp_project.h"

namespace lfbp {

// Status word of the library on each device: 0 or a negative LFBP_ERR_* code
// written by a kernel whose bounded wait gave up.
__device__ int g_status;


constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per in-kernel wait
constexpr int kPlainThreads = 256;
constexpr int kProducerWarps = 2;  // warps sharing each tile's bulk copies
constexpr int kConsumerWarps = 7;
constexpr int kPersistentThreads = 32 * (kProducerWarps + kConsumerWarps);
// Per-stage info slot: [16 B: end flag (persistent) or mbarrier (plain)]
// [TileCtx][row-base table: kMaxTileRows + 1 ints]
constexpr int kCtxBytes = (int)((sizeof(TileCtx) + 15) / 16 * 16);
constexpr int kTabBytes = (4 * (kMaxTileRows + 1) + 15) / 16 * 16;
constexpr int kInfoBytes = 16 + kCtxBytes + kTabBytes;
constexpr int kStatusBadLaunch = -9;  // LFBP_ERR_INVALID: launched with too little shared memory

// Dynamic shared memory of the plain kernel for a stage of `stage_bytes`:
// [stage][mbarrier, 16 B][TileCtx][row-base table].
__host__ __device__ constexpr int plain_smem_bytes(int stage_bytes) {
  return stage_bytes + kInfoBytes;
}
// ... and of the persistent kernel: [stages][per-stage info][full, empty barriers].
__host__ __device__ constexpr int persistent_smem_bytes(int stage_bytes, int nstages) {
  return nstages * (stage_bytes + kInfoBytes) + nstages * 16;
}

__device__ __forceinline__ uint32_t dynamic_smem_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

// ------------------------------------------------------------------ plain --
// grid = (nV, Nx, nU) tiles of one depth; block = kPlainThreads; one tile per
// CTA.  `base` carries the depth's shape, pitch and flags; the CTA fills in
// its own p, u0, v0, nrows, ncols.
// smem: [stage: tile bytes][mbarrier][TileCtx][row-base table]
// The four tile shapes of one depth: index (last row block) + 2 (last column block).
struct DepthShapes {
  TileShape s[4];
};

// Register cap of the one-tile-per-CTA kernels: 48 registers (room for 5 CTAs
// of 256 threads per SM).  Measured against the uncapped 61 registers, per-depth
// graph: highres fp32 6080 -> 6273 GB/s, Table 1 N = 51 4709 -> 5692, fp16
// 5330 -> 5410 (at 40 registers, 6 CTAs, the spills cost more than the warps
// gain).
constexpr int kPlainMinBlocks = 5;

__global__ void __launch_bounds__(kPlainThreads, kPlainMinBlocks)
    k_gather_depth(TileDesc base, const __grid_constant__ DepthShapes shapes,
                   const unsigned char* __restrict__ in_depth, const unsigned char* in_safe_end,
                   unsigned char* __restrict__ out_depth, int J, int V, int stage_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stage = smem;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_bytes);
  TileCtx* ctx = reinterpret_cast<TileCtx*>(smem + stage_bytes + 16);
  int* tab = reinterpret_cast<int*>(smem + stage_bytes + 16 + kCtxBytes);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (dynamic_smem_size() < (uint32_t)plain_smem_bytes(stage_bytes)) {
    if (tid == 0) set_status(kStatusBadLaunch);
    return;
  }

  TileDesc td = base;
  td.p = (unsigned short)blockIdx.y;
  const int u0 = blockIdx.z * J, v0 = blockIdx.x * V;
  td.u0 = (unsigned short)u0;
  td.v0 = (unsigned short)v0;
  td.nrows = (unsigned short)min(J, (int)base.Ks - u0);
  td.ncols = (unsigned short)min(V, (int)base.Kt - v0);

  const uint32_t b = smem_addr(bar);
  constexpr int kWarps = kPlainThreads / 32;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(b, kWarps);
    fence_mbar_init();
  }
  __syncthreads();
  // every warp issues a share of the tile's copies; the tile context is built
  // while they are in flight; then all wait for them
  issue_tile_loads(td, in_depth, in_safe_end, stage, b, lane, warp, kWarps);
  __syncwarp();
  if (lane == 0) mbar_arrive(b);
  // the tile context: warp 0 copies the shape record, warps 1..4 each build
  // one part of the tile fields (in parallel)
  {
    const int si = (blockIdx.z + 1 == gridDim.z ? 1 : 0) + (blockIdx.x + 1 == gridDim.x ? 2 : 0);
    const TileShape* shp = &shapes.s[si];
    if (warp == 0) copy_shape(*ctx, shp, lane);
    if (warp >= 1 && warp <= 4 && lane == 0)
      make_ctx_tile(*ctx, td, shp, stage, in_depth, out_depth, tab, warp - 1);
  }
  __syncthreads();
  if (!mbar_wait_bounded(b, 0, &abort_flag, kWaitLimitNs)) {
    set_status(kStatusTimeout);
    abort_flag = 1;
    // give the copies in flight a last bounded chance to land before exit
    mbar_wait_bounded(b, 0, nullptr, kWaitLimitNs);
    return;
  }
  gather_tile_ctx(*ctx, warp, kPlainThreads / 32, lane);
}

// ------------------------------------------------------------------ tiles --
// The batched form with one tile of the work list per CTA: grid = ntiles,
// block = kPlainThreads, the body of k_gather_depth (every warp issues a share
// of the tile's copies, the context is built while they are in flight, then
// every warp gathers).  The hardware block scheduler overlaps the CTAs of an
// SM that wait for their copies with those that gather.
// smem: [stage: stage_bytes][mbarrier][TileCtx][row-base table]
__global__ void __launch_bounds__(kPlainThreads, kPlainMinBlocks)
    k_gather_tiles(const __grid_constant__ BatchPtrs ptrs, const TileDesc* __restrict__ tiles,
                   const TileShape* __restrict__ shapes, int stage_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stage = smem;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_bytes);
  TileCtx* ctx = reinterpret_cast<TileCtx*>(smem + stage_bytes + 16);
  int* tab = reinterpret_cast<int*>(smem + stage_bytes + 16 + kCtxBytes);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (dynamic_smem_size() < (uint32_t)plain_smem_bytes(stage_bytes)) {
    if (tid == 0) set_status(kStatusBadLaunch);
    return;
  }
  const TileDesc td = tiles[blockIdx.x];
  const unsigned char* in_arr = ptrs.in[td.arr];
  const unsigned char* in_depth = in_arr + td.off_bytes;
  const unsigned char* safe_end = in_arr + (ptrs.in_bytes[td.arr] & ~15ull);
  unsigned char* out_depth = ptrs.out[td.arr] + td.off_bytes;

  const uint32_t b = smem_addr(bar);
  constexpr int kWarps = kPlainThreads / 32;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(b, kWarps);
    fence_mbar_init();
  }
  __syncthreads();
  issue_tile_loads(td, in_depth, safe_end, stage, b, lane, warp, kWarps);
  __syncwarp();
  if (lane == 0) mbar_arrive(b);
  {
    const TileShape* shp = shapes + td.shape;
    if (warp == 0) copy_shape(*ctx, shp, lane);
    if (warp >= 1 && warp <= 4 && lane == 0)
      make_ctx_tile(*ctx, td, shp, stage, in_depth, out_depth, tab, warp - 1);
  }
  __syncthreads();
  if (!mbar_wait_bounded(b, 0, &abort_flag, kWaitLimitNs)) {
    set_status(kStatusTimeout);
    abort_flag = 1;
    mbar_wait_bounded(b, 0, nullptr, kWaitLimitNs);
    return;
  }
  gather_tile_ctx(*ctx, warp, kWarps, lane);
}

// ------------------------------------------------------------- persistent --
// grid = SMs * ctas_per_sm; block = kPersistentThreads.  CTA c takes tiles
// c, c + grid, c + 2 grid, ... (consecutive tiles are neighbours in memory, so
// the tiles in flight at any time cover one contiguous stretch of the work
// list).  Warps 0 .. kProducerWarps-1 produce: each prefetches the next
// descriptor, waits for a free stage and issues its share of the stage's bulk
// copies (warp 0 also writes the stage's tile context); the other warps
// consume.
// smem: [nstages x stage_bytes][nstages x descriptor][full[nstages]][empty[nstages]]
//
// kStall (fault injection for tests of the error paths, LFBP_FAULT=stall):
// the producers register their copies' bytes on the full barrier without
// issuing the copies, so no barrier phase completes, every consumer wait runs
// out and the kernel ends with LFBP_ERR_TIMEOUT in the status word.  The
// normal instantiation is kStall = false.
// kLsu: the producers move the segments with 16-byte cp.async copies
// (tile_copies_lsu) instead of TMA bulk copies; every producer lane then
// arrives on the stage's full barrier once its copies have landed, so that
// barrier counts 32 * kProducerWarps + kProducerWarps arrivals.  Used for
// inputs in host memory, and for device inputs where it is faster.
template <bool kStall, bool kLsu = false>
#ifndef LFBP_PERSIST_MINB
#define LFBP_PERSIST_MINB 3
#endif
__global__ void __launch_bounds__(kPersistentThreads, LFBP_PERSIST_MINB)
    k_gather_persistent(const __grid_constant__ BatchPtrs ptrs,
                        const TileDesc* __restrict__ tiles, const TileShape* __restrict__ shapes,
                        int ntiles, int stage_bytes, int nstages) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* info_base = smem + (size_t)nstages * stage_bytes;  // per stage: flag, TileCtx, table
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstages * (stage_bytes + kInfoBytes));
  uint64_t* empty = full + nstages;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (dynamic_smem_size() < (uint32_t)persistent_smem_bytes(stage_bytes, nstages)) {
    if (tid == 0) set_status(kStatusBadLaunch);
    return;
  }

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_addr(&full[s]), kLsu ? 33 * kProducerWarps : kProducerWarps);
      mbar_init(smem_addr(&empty[s]), kConsumerWarps);
      // the shape index held by the stage's context slot: none yet
      reinterpret_cast<int*>(info_base + (size_t)s * kInfoBytes)[1] = -1;
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp < kProducerWarps) {
    // ---- producer warps
    int it = 0;
    int t = blockIdx.x;
    TileDesc td;
    if (t < ntiles) td = tiles[t];
    for (;; ++it, t += gridDim.x) {
      const int s = it % nstages;
      const uint32_t fb = smem_addr(&full[s]);
      TileDesc next;
      const int tn = t + (int)gridDim.x;
      if (tn < ntiles) next = tiles[tn];  // in flight while this tile is issued
      if (it >= nstages) {
        const uint32_t par = (uint32_t)((it / nstages - 1) & 1);
        if (!mbar_wait_bounded(smem_addr(&empty[s]), par, &abort_flag, kWaitLimitNs)) {
          if (lane == 0) {
            set_status(kStatusTimeout);
            abort_flag = 1;
          }
          break;
        }
      }
      if (t >= ntiles) {
        if (kLsu) cp_async_arrive_noinc(fb);  // no copies pending: arrives at once
        if (lane == 0) {
          if (warp == 0) *reinterpret_cast<int*>(info_base + (size_t)s * kInfoBytes) = 1;  // end of work
          mbar_arrive(fb);
        }
        ++it;
        break;
      }
      const unsigned char* in_arr = ptrs.in[td.arr];
      const unsigned char* in_depth = in_arr + td.off_bytes;
      const unsigned char* safe_end = in_arr + (ptrs.in_bytes[td.arr] & ~15ull);
      if (kStall) {
        if (lane == 0) mbar_expect_tx(fb, 16);
      } else if (kLsu) {
        tile_copies_lsu(td, in_depth, safe_end, smem + (size_t)s * stage_bytes, lane, warp,
                        kProducerWarps);
        cp_async_arrive_noinc(fb);
      } else {
        issue_tile_loads(td, in_depth, safe_end, smem + (size_t)s * stage_bytes, fb, lane, warp,
                         kProducerWarps);
      }
      // the tile context, built by warp 0 while the copies are in flight: the
      // shape record is copied only when the slot holds another one (the tiles
      // of one CTA come from one depth for long stretches), then lanes 0..3
      // build the tile fields from the slot's copy of the shape
      if (warp == 0) {
        unsigned char* info = info_base + (size_t)s * kInfoBytes;
        TileCtx& ctx = *reinterpret_cast<TileCtx*>(info + 16);
        int* held = reinterpret_cast<int*>(info) + 1;
        if (lane == 0) reinterpret_cast<int*>(info)[0] = 0;
        if (*held != (int)td.shape) {
          copy_shape(ctx, shapes + td.shape, lane);
          __syncwarp();
          if (lane == 0) *held = td.shape;
        }
        __syncwarp();
        if (lane < 4)
          make_ctx_tile(ctx, td, &ctx, smem + (size_t)s * stage_bytes, in_depth,
                        ptrs.out[td.arr] + td.off_bytes,
                        reinterpret_cast<int*>(info + 16 + kCtxBytes), lane);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(fb);
      td = next;
    }
    // make sure no copy into this CTA's shared memory is still in flight (the
    // full barriers count the bytes of every producer warp's copies; cp.async
    // copies are waited for by the lane that issued them)
    if (kLsu) cp_async_wait_all();
    if (lane == 0 && !kStall && !kLsu) {
      const int armed = it;  // stages armed: iterations 0..it-1
      for (int s = 0; s < nstages && s < armed; ++s) {
        const int last = ((armed - 1 - s) / nstages) * nstages + s;  // last iteration using s
        const uint32_t par = (uint32_t)((last / nstages) & 1);
        mbar_wait_bounded(smem_addr(&full[s]), par, nullptr, kWaitLimitNs);
      }
    }
  } else {
    // ---- consumer warps
    const int cw = warp - kProducerWarps;
    for (int it = 0;; ++it) {
      const int s = it % nstages;
      const uint32_t par = (uint32_t)((it / nstages) & 1);
      if (!mbar_wait_bounded(smem_addr(&full[s]), par, &abort_flag, kWaitLimitNs)) {
        if (lane == 0) {
          set_status(kStatusTimeout);
          abort_flag = 1;
        }
        break;
      }
      const unsigned char* info = info_base + (size_t)s * kInfoBytes;
      if (*reinterpret_cast<const int*>(info) != 0) break;
      // rotate the step-to-warp assignment by the tile's step count
      const TileCtx& tc = *reinterpret_cast<const TileCtx*>(info + 16);
      const int nsteps = tc.pair ? (tc.punits + 31) / 32
                                 : (tc.stripe ? tc.nsteps_s : (tc.fast ? tc.nunits : tc.items));
      gather_tile_ctx(tc, cw, kConsumerWarps, lane, (it * nsteps) % kConsumerWarps);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
    }
  }
}

}  // namespace lfbp

// ====================================================================== host
#include <cmath>

#include "lfbp_host_sched.h"

using namespace lfbp;

struct lfbp_plan_s {
  int Nx = 0, Ny = 0, Nz = 0;
  std::vector<int> Ks, Kt;
  lfbp_dtype dt = LFBP_F32;
  lfbp_mode mode = LFBP_MAP_TRANSPOSE;
  int es = 4;
  std::vector<size_t> off;  // Nz + 1
  unsigned long long uid = 0;
  // an even cut-out (paper-window mode only): the map is the literal
  // Eqs. (4)-(9) loop, which the gather runs as the cropped odd cut-out
  // under the loop ranges' window; the projectors need odd cut-outs
  bool literal = false;
  // per-depth tilings by tile-size target (built lazily; entries stay put)
  std::mutex mu;
  std::map<int, std::vector<lfbp::DepthTiling>> tilings;
};

namespace {

thread_local std::string t_err;

int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LFBP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::mutex g_mu;
unsigned long long g_next_uid = 1;

// LFBP_FAULT: plan | alloc | graph | stall -- injected failures for tests of
// the error paths (plan creation, the work list's device allocation, the
// graph instantiation, a persistent kernel whose waits run out).
enum Fault { kFaultNone = 0, kFaultPlan, kFaultAlloc, kFaultGraph, kFaultStall };
int fault_mode() {
  const char* s = std::getenv("LFBP_FAULT");
  if (!s || !*s) return kFaultNone;
  if (!std::strcmp(s, "plan")) return kFaultPlan;
  if (!std::strcmp(s, "alloc")) return kFaultAlloc;
  if (!std::strcmp(s, "graph")) return kFaultGraph;
  if (!std::strcmp(s, "stall")) return kFaultStall;
  return kFaultNone;
}

int env_int(const char* name, int dflt) {
  const char* s = std::getenv(name);
  if (!s || !*s) return dflt;
  return std::atoi(s);
}

// Launch-shape knobs (set by the tuner or the environment).
struct Tuning {
  int tile_bytes;   // target shared-memory bytes of one tile
  int ctas_per_sm;  // persistent CTAs per SM
  int stages;       // stages per persistent CTA (0 = as many as fit)
  int pairs;        // 1: tiles that can take the pair consumer do (lfbp_pairs.cuh)
  int form;         // 0: persistent CTAs (k_gather_persistent); 1: one tile per CTA (k_gather_tiles)
};

// Untuned launch shape: one tile per CTA with 64 KB tiles (measured the most
// even across the workloads: highres fp32 5696, fp16 5227, mid 5821, Table 1
// N = 51 5215, 95 x 55 5777 GB/s; persistent CTAs with 32 KB tiles, the
// default before, 5577 / 4615 / 5185 / 4095 / 3809).  The graph of per-depth
// grids is faster on few large depths (highres fp32 6296) but pays a launch
// per node on many small ones (mid 2929): the autotuner chooses per batch.
Tuning default_tuning() {
  Tuning t;
  t.form = std::min(2, std::max(0, env_int("LFBP_FORM", 1)));
  t.tile_bytes = env_int("LFBP_TILE_BYTES", t.form == 0 ? 32768 : 65536);
  t.ctas_per_sm = env_int("LFBP_CTAS_PER_SM", 3);
  t.stages = env_int("LFBP_STAGES", 0);
  t.pairs = env_int("LFBP_PAIRS", 1) != 0;
  if (t.tile_bytes < 1024) t.tile_bytes = 1024;
  if (t.tile_bytes > 65536) t.tile_bytes = 65536;
  if (t.ctas_per_sm < 1) t.ctas_per_sm = 1;
  if (t.ctas_per_sm > 4) t.ctas_per_sm = 4;
  return t;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

int check_buffers(lfbp_plan p, const void* in, const void* out) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  const size_t bytes = p->off.back() * (size_t)p->es;
  if (bytes == 0) return LFBP_OK;
  if (!in || !out) return fail(LFBP_ERR_NULL, "buffer pointer is NULL");
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15))
    return fail(LFBP_ERR_ALIGN, "buffers must start on a 16-byte boundary");
  if (overlaps(in, bytes, out, bytes)) return fail(LFBP_ERR_ALIAS, "input and output overlap");
  return LFBP_OK;
}

int ensure_smem_attr(const void* fn, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  return LFBP_OK;
}

int device_props(int* dev, int* sms, int* smem_optin) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  e = cudaDeviceGetAttribute(smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, *dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  return LFBP_OK;
}

// Per-depth tiling of a plan for a tile-size target, cached in the plan.
const std::vector<DepthTiling>& plan_tiling(lfbp_plan p, int target) {
  std::lock_guard<std::mutex> lk(p->mu);
  std::vector<DepthTiling>& t = p->tilings[target];
  if ((int)t.size() != p->Nz) {
    t.clear();
    for (int z = 0; z < p->Nz; ++z) t.push_back(tile_depth(p->Ny, p->Ks[z], p->Kt[z], p->es, target));
  }
  return t;
}

// pairs = 0 keeps the depth's tiles off the pair consumer (flags bit 5).
TileDesc depth_desc(lfbp_plan p, int z, const DepthTiling& d, int mode, int arr, int pairs) {
  TileDesc t;
  std::memset(&t, 0, sizeof(t));
  t.off_bytes = p->off[z] * (size_t)p->es;
  t.Nx = (unsigned short)p->Nx;
  t.Ny = (unsigned short)p->Ny;
  t.Ks = (unsigned short)p->Ks[z];
  t.Kt = (unsigned short)p->Kt[z];
  t.P = (unsigned short)d.P;
  t.arr = (unsigned char)arr;
  t.flags = (unsigned char)((p->es == 2 ? 1 : 0) | (mode << 1) | ((p->Ks[z] % 2 == 0) << 3) |
                            ((p->Kt[z] % 2 == 0) << 4) | (pairs ? 0 : 32));
  return t;
}

// The four tile shapes of depth z for a tiling: index (last row block) +
// 2 (last column block).
void depth_shapes(lfbp_plan p, int z, const DepthTiling& d, const TileDesc& base, TileShape* out) {
  for (int cls = 0; cls < 4; ++cls)
    out[cls] = depth_shape(d, p->Nx, p->Ny, p->Ks[z], p->Kt[z], p->es, base.flags, cls);
}

// One launch per depth of the plain kernel, for depths [z0, z1).
// Tile-size target of the plain form: one tile per CTA and no pipeline, so
// larger tiles than the persistent form's pay (measured on highres: 64 KB
// 4705 GB/s, 48 KB 4535, 32 KB 4390).
int plain_tile_bytes() {
  int t = env_int("LFBP_PLAIN_TILE_BYTES", 65536);
  return t < 1024 ? 1024 : (t > 65536 ? 65536 : t);
}

// Helper streams of the plain form, per device: consecutive depth launches go
// round-robin to kPlainStreams streams forked from the caller's stream and
// joined back into it, so that a depth too small to fill the GPU runs beside
// its neighbours (each depth is still one launch).
constexpr int kPlainStreams = 4;
struct PlainStreams {
  int dev = -1;
  std::mutex mu;  // held from the fork to the join of one call
  cudaStream_t s[kPlainStreams] = {};
  cudaEvent_t fork = nullptr, join[kPlainStreams] = {};
};
std::vector<PlainStreams*> g_plain_streams;  // guarded by g_mu; live as long as the process

PlainStreams* plain_streams() {
  if (env_int("LFBP_PLAIN_STREAMS", 1) == 0) return nullptr;  // 0: the caller's stream only
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  for (PlainStreams* s : g_plain_streams)
    if (s->dev == dev) return s;
  PlainStreams* s = new PlainStreams();
  s->dev = dev;
  bool ok = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < kPlainStreams; ++i)
    ok = cudaStreamCreateWithFlags(&s->s[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {  // a partly created set is dropped; launches stay on the caller's stream
    cudaGetLastError();
    return nullptr;
  }
  g_plain_streams.push_back(s);
  return s;
}

int launch_plain(lfbp_plan p, const unsigned char* inb, unsigned char* outb, int mode, int z0,
                 int z1, cudaStream_t st) {
  const size_t arr_bytes = p->off.back() * (size_t)p->es;
  const unsigned char* safe_end = inb + (arr_bytes & ~(size_t)15);
  const std::vector<DepthTiling>& tl = plan_tiling(p, plain_tile_bytes());
  int max_smem = 0;
  for (int z = z0; z < z1; ++z) max_smem = std::max(max_smem, tl[z].max_tile_bytes);
  int rc = ensure_smem_attr((const void*)k_gather_depth, plain_smem_bytes((max_smem + 15) & ~15));
  if (rc) return rc;
  PlainStreams* ps = z1 - z0 > 1 ? plain_streams() : nullptr;
  std::unique_lock<std::mutex> ps_lock;
  if (ps) {
    ps_lock = std::unique_lock<std::mutex>(ps->mu);
    cudaError_t e = cudaEventRecord(ps->fork, st);
    for (int i = 0; e == cudaSuccess && i < kPlainStreams; ++i)
      e = cudaStreamWaitEvent(ps->s[i], ps->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "plain-form fork");
  }
  for (int z = z0; z < z1; ++z) {
    cudaStream_t sz = ps ? ps->s[(z - z0) % kPlainStreams] : st;
    const DepthTiling& d = tl[z];
    // the pair consumer measured faster for fp16 plain launches, slower for fp32
    const TileDesc base = depth_desc(p, z, d, mode, 0, p->es == 2);
    DepthShapes ds;
    depth_shapes(p, z, d, base, ds.s);
    dim3 grid(d.nV, p->Nx, d.nU);
    const int smem = (d.max_tile_bytes + 15) & ~15;
    k_gather_depth<<<grid, kPlainThreads, plain_smem_bytes(smem), sz>>>(
        base, ds, inb + base.off_bytes, safe_end, outb + base.off_bytes, d.J, d.V, smem);
  }
  cudaError_t e = cudaGetLastError();
  if (ps) {  // join: later work on st waits for every depth
    const int used = std::min(kPlainStreams, z1 - z0);
    for (int i = 0; i < used; ++i) {
      cudaError_t e2 = cudaEventRecord(ps->join[i], ps->s[i]);
      if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, ps->join[i], 0);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "k_gather_depth launch");
  return LFBP_OK;
}

int run_plain(lfbp_plan p, const void* in, void* out, int mode, cudaStream_t st) {
  int rc = check_buffers(p, in, out);
  if (rc) return rc;
  if (p->off.back() == 0) return LFBP_OK;  // an empty plan: no CUDA call at all
  return launch_plain(p, (const unsigned char*)in, (unsigned char*)out, mode, 0, p->Nz, st);
}

// True when no array of the batch has an element.
bool batch_empty(int n, const lfbp_plan* plans) {
  for (int i = 0; i < n; ++i)
    if (plans[i]->off.back() != 0) return false;
  return true;
}

// --------------------------------------------------- host-to-host pipeline --
// Per device: two helper streams and a pool of events for overlapping the
// host->device copy of depth chunk c+1, the map of chunk c on the caller's
// stream and the device->host copy of chunk c-1.
struct HostPipe {
  int dev = -1;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  std::vector<cudaEvent_t> ev;
  std::mutex mu;
  ~HostPipe() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (h2d) cudaStreamDestroy(h2d);
    if (d2h) cudaStreamDestroy(d2h);
  }
};
std::vector<std::unique_ptr<HostPipe>> g_pipes;  // guarded by g_mu

int get_pipe(int dev, HostPipe** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pipes)
    if (p->dev == dev) {
      *out = p.get();
      return LFBP_OK;
    }
  std::unique_ptr<HostPipe> hp(new HostPipe());
  hp->dev = dev;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  if ((e = cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  *out = hp.get();
  g_pipes.push_back(std::move(hp));
  return LFBP_OK;
}

// Device address of a host buffer of `bytes` bytes that the current device can
// read and write directly (page-locked and mapped: cudaHostAlloc,
// cudaHostRegister, or torch's pinned tensors), or nullptr.  The buffer must
// also be 16-byte aligned, as every array of the map.
void* mapped_host_ptr(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // clear the error of a pointer the runtime does not know
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  if ((uintptr_t)a.devicePointer & 15) return nullptr;
  return a.devicePointer;
}

// Host-to-host path: LFBP_HOST_PATH=zerocopy lets the kernel read and write
// mapped host buffers itself (read at each call); the default stages aligned
// chunks through the device buffers, which measured faster (23.8 against
// 34.8 ms per highres step: the zero-copy kernel's 1.6 KB pieces scattered
// over host memory run below the link's rate).
bool env_zero_copy() {
  const char* s = std::getenv("LFBP_HOST_PATH");
  return s && !std::strcmp(s, "zerocopy");
}

int run_batched(int n, const lfbp_plan* plans, const void* const* in, void* const* out,
                cudaStream_t st, int lsu_force);

int run_host(lfbp_plan p, const void* H_host, void* Hp_host, void* dH, void* dHp, int mode,
             cudaStream_t st) {
  int rc = check_buffers(p, dH, dHp);
  if (rc) return rc;
  const size_t bytes = p->off.back() * (size_t)p->es;
  if (bytes == 0) return LFBP_OK;
  if (!H_host || !Hp_host) return fail(LFBP_ERR_NULL, "host buffer pointer is NULL");
  if (overlaps(H_host, bytes, Hp_host, bytes))
    return fail(LFBP_ERR_ALIAS, "host input and output overlap");
  // Zero-copy (opt-in): both buffers page-locked and mapped, the persistent
  // kernel reads H from host memory and writes H' to host memory itself (one
  // launch; loads by cp.async through the load/store path, not TMA); the
  // device work buffers are not touched.
  if (env_zero_copy()) {
    void* din = mapped_host_ptr(H_host);
    void* dout = din ? mapped_host_ptr(Hp_host) : nullptr;
    if (din && dout) {
      const void* ins[1] = {din};
      void* outs[1] = {dout};
      return run_batched(1, &p, ins, outs, st, 1);
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  HostPipe* hp = nullptr;
  if ((rc = get_pipe(dev, &hp))) return rc;
  // The copies move fixed byte ranges of LFBP_HOST_CHUNK_MB (default 64) MB,
  // cut at multiples of the chunk size whatever the depth boundaries (copies
  // from and to aligned addresses run at the link's rate; copies cut at depth
  // starts, which are only 4-byte aligned, measured 25 % slower).  A depth is
  // mapped once every chunk it overlaps has arrived, and a chunk is copied back
  // once every depth overlapping it is mapped.  host_schedule gives the order:
  // the depths in memory order (LFBP_HOST_ORDER=rotate: a rotation that starts
  // and ends on small depths, which measured slower).
  // (Holding copy k in until copy k - 2 or k - 1 is back measured 2-3 x slower:
  // a depth spanning several ranges holds its ranges back until its last one
  // has arrived.)
  const size_t chunk = (size_t)std::max(1, env_int("LFBP_HOST_CHUNK_MB", 64)) << 20;
  const int nch = (int)((bytes + chunk - 1) / chunk);
  const char* ord = std::getenv("LFBP_HOST_ORDER");
  std::vector<size_t> zoff(p->Nz + 1);
  for (int z = 0; z <= p->Nz; ++z) zoff[z] = p->off[z] * (size_t)p->es;
  const std::vector<HostOp> ops = host_schedule(zoff, chunk, !(ord && !std::strcmp(ord, "rotate")));
  std::lock_guard<std::mutex> lk(hp->mu);
  while ((int)hp->ev.size() < 2 * nch + 2) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    hp->ev.push_back(ev);
  }
  // events: in[k] = ev[k]; the j-th release of copies back ev[nch + j] (at
  // most nch: each releases a chunk); start ev[2 nch]; end ev[2 nch + 1]
  const unsigned char* hin = (const unsigned char*)H_host;
  unsigned char* hout = (unsigned char*)Hp_host;
  unsigned char* din = (unsigned char*)dH;
  unsigned char* dout = (unsigned char*)dHp;
  cudaEvent_t start = hp->ev[2 * nch], end = hp->ev[2 * nch + 1];
  if ((e = cudaEventRecord(start, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(hp->h2d, start, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamWaitEvent");
  std::vector<int> pos(nch, -1);  // issue position of each copy in
  int issued = 0, waited = -1;    // copies in issued; position the caller's stream waited for
  int releases = 0;
  bool mapped_since_release = false;
  for (const HostOp& op : ops) {
    const size_t o = (size_t)op.a * chunk, n = std::min(chunk, bytes - o);
    if (op.kind == HostOp::kIn) {
      if ((e = cudaMemcpyAsync(din + o, hin + o, n, cudaMemcpyHostToDevice, hp->h2d)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(H2D)");
      if ((e = cudaEventRecord(hp->ev[op.a], hp->h2d)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
      pos[op.a] = issued++;
    } else if (op.kind == HostOp::kMap) {
      if (pos[op.wait] > waited) {  // copies in land in issue order
        if ((e = cudaStreamWaitEvent(st, hp->ev[op.wait], 0)) != cudaSuccess)
          return cuda_fail(e, "cudaStreamWaitEvent");
        waited = pos[op.wait];
      }
      if ((rc = launch_plain(p, din, dout, mode, op.a, op.b, st))) return rc;
      mapped_since_release = true;
    } else {
      if (mapped_since_release) {
        cudaEvent_t rel = hp->ev[nch + releases++];
        if ((e = cudaEventRecord(rel, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(hp->d2h, rel, 0)) != cudaSuccess)
          return cuda_fail(e, "cudaStreamWaitEvent");
        mapped_since_release = false;
      }
      if ((e = cudaMemcpyAsync(hout + o, dout + o, n, cudaMemcpyDeviceToHost, hp->d2h)) !=
          cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
  }
  // the caller's stream sees the whole call complete: the last copy back, and
  // (by stream order) every map launched on it
  if ((e = cudaEventRecord(end, hp->d2h)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  if ((e = cudaStreamWaitEvent(st, end, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamWaitEvent");
  return LFBP_OK;
}

// ---------------------------------------------------------------- batched --
// One depth of one array in the form-2 graph (k_gather_depth's arguments
// apart from the pointers, which come from the batch's pointers at launch).
struct DepthNode {
  TileDesc base;    // arr, off_bytes, sizes, pitch, flags
  DepthShapes ds;
  dim3 grid;
  int J = 0, V = 0, stage = 0;
};
struct DepthNodeArgs {  // storage for one node's kernel arguments
  TileDesc base;
  DepthShapes ds;
  const unsigned char* in = nullptr;
  const unsigned char* safe_end = nullptr;
  unsigned char* out = nullptr;
  int J = 0, V = 0, stage = 0;
  void* args[8];
};

struct BatchState {
  int dev = -1;
  bool lsu = false;  // producers move the segments with cp.async (k_gather_persistent<false, true>)
  int form = 0;      // 0: k_gather_persistent; 1: k_gather_tiles (one tile per CTA);
                     // 2: a graph of k_gather_depth grids, one per depth of every array
  std::vector<DepthNode> dnodes;         // form 2: the depths
  std::vector<cudaGraphNode_t> knodes;   // form 2: their graph nodes
  std::vector<unsigned long long> uids;
  Tuning tuning{0, 0, 0, 0, 0};
  int ntiles = 0;
  int stage_bytes = 0, nstages = 0, grid = 0, smem = 0;
  TileDesc* d_tiles = nullptr;    // work list, followed in the same allocation by
  TileShape* d_shapes = nullptr;  // the shape table
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  BatchPtrs ptrs;
  unsigned long long last_use = 0;
  ~BatchState() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_tiles) cudaFree(d_tiles);
  }
};

std::vector<std::unique_ptr<BatchState>> g_batches;  // guarded by g_mu

// Launch shapes chosen by lfbp_tune_batched, per list of plans (by uid).
struct TunedEntry {
  int dev;
  std::vector<unsigned long long> uids;
  Tuning tuning;
};
std::vector<TunedEntry> g_tuned;  // guarded by g_mu

bool same_uids(const std::vector<unsigned long long>& u, int n, const lfbp_plan* plans) {
  if ((int)u.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (u[i] != plans[i]->uid) return false;
  return true;
}

Tuning tuning_for(int dev, int n, const lfbp_plan* plans) {
  for (const TunedEntry& t : g_tuned)
    if (t.dev == dev && same_uids(t.uids, n, plans)) return t.tuning;
  return default_tuning();
}
unsigned long long g_clock = 0;
constexpr size_t kMaxCachedBatches = 8;

// Work list of all depths of all arrays: per depth, u-block major, then p,
// then v-block, so that tiles in flight together touch neighbouring input
// segments and neighbouring output runs.
// With each depth come its four tile shapes (depth_shapes), referenced by index.
void build_tiles(int n, const lfbp_plan* plans, int target, int pairs, std::vector<TileDesc>& tiles,
                 std::vector<TileShape>& shapes, int* max_tile) {
  *max_tile = 0;
  for (int i = 0; i < n; ++i) {
    lfbp_plan p = plans[i];
    const std::vector<DepthTiling>& tl = plan_tiling(p, target);
    for (int z = 0; z < p->Nz; ++z) {
      const DepthTiling& d = tl[z];
      *max_tile = std::max(*max_tile, d.max_tile_bytes);
      const TileDesc base = depth_desc(p, z, d, (int)p->mode, i, pairs);
      const size_t s0 = shapes.size();
      shapes.resize(s0 + 4);
      depth_shapes(p, z, d, base, &shapes[s0]);
      for (int ub = 0; ub < d.nU; ++ub)
        for (int pp = 0; pp < p->Nx; ++pp)
          for (int vb = 0; vb < d.nV; ++vb) {
            TileDesc t = base;
            t.shape = (unsigned short)(s0 + (ub + 1 == d.nU ? 1 : 0) + (vb + 1 == d.nV ? 2 : 0));
            t.p = (unsigned short)pp;
            t.u0 = (unsigned short)(ub * d.J);
            t.v0 = (unsigned short)(vb * d.V);
            t.nrows = (unsigned short)std::min(d.J, p->Ks[z] - ub * d.J);
            t.ncols = (unsigned short)std::min(d.V, p->Kt[z] - vb * d.V);
            tiles.push_back(t);
          }
    }
  }
}

// The persistent kernel's entry for a batch: TMA bulk copies, or cp.async
// copies through the load/store path.
const void* persistent_fn(bool lsu) {
  return lsu ? (const void*)k_gather_persistent<false, true>
             : (const void*)k_gather_persistent<false, false>;
}

// Which copy path device-resident batches use: LFBP_LOADS=lsu or tma (default),
// read at each call.
bool env_lsu() {
  const char* s = std::getenv("LFBP_LOADS");
  return s && !std::strcmp(s, "lsu");
}

// The kernel of a batch, and its graph node's launch parameters (args: room
// for 6 pointers, kept alive by the caller until the node is set).
const void* batch_fn(const BatchState& bs) {
  return bs.form == 1 ? (const void*)k_gather_tiles : persistent_fn(bs.lsu);
}
void batch_node_params(BatchState& bs, void** args, cudaKernelNodeParams* kp) {
  std::memset(kp, 0, sizeof(*kp));
  args[0] = &bs.ptrs;
  args[1] = &bs.d_tiles;
  args[2] = &bs.d_shapes;
  if (bs.form == 1) {
    args[3] = &bs.stage_bytes;
    kp->blockDim = dim3(kPlainThreads);
  } else {
    args[3] = &bs.ntiles;
    args[4] = &bs.stage_bytes;
    args[5] = &bs.nstages;
    kp->blockDim = dim3(kPersistentThreads);
  }
  kp->func = (void*)batch_fn(bs);
  kp->gridDim = dim3(bs.grid);
  kp->sharedMemBytes = bs.smem;
  kp->kernelParams = args;
}

// Sets the launch parameters of a depth node (form 2) for the batch's
// pointers: the k_gather_depth arguments of one depth of one array.
void depth_node_params(const BatchState& bs, const DepthNode& dn, DepthNodeArgs& a,
                       cudaKernelNodeParams* kp) {
  a.base = dn.base;
  a.ds = dn.ds;
  const unsigned char* in_arr = bs.ptrs.in[dn.base.arr];
  a.in = in_arr ? in_arr + dn.base.off_bytes : nullptr;
  a.safe_end = in_arr ? in_arr + (bs.ptrs.in_bytes[dn.base.arr] & ~15ull) : nullptr;
  a.out = bs.ptrs.out[dn.base.arr] ? bs.ptrs.out[dn.base.arr] + dn.base.off_bytes : nullptr;
  a.J = dn.J;
  a.V = dn.V;
  a.stage = dn.stage;
  a.args[0] = &a.base;
  a.args[1] = &a.ds;
  a.args[2] = &a.in;
  a.args[3] = &a.safe_end;
  a.args[4] = &a.out;
  a.args[5] = &a.J;
  a.args[6] = &a.V;
  a.args[7] = &a.stage;
  std::memset(kp, 0, sizeof(*kp));
  kp->func = (void*)k_gather_depth;
  kp->gridDim = dn.grid;
  kp->blockDim = dim3(kPlainThreads);
  kp->sharedMemBytes = plain_smem_bytes(dn.stage);
  kp->kernelParams = a.args;
}

int build_batch(BatchState& bs, int n, const lfbp_plan* plans, const Tuning& tu) {
  int sms = 0, optin = 0, dev = 0;
  int rc = device_props(&dev, &sms, &optin);
  if (rc) return rc;
  bs.dev = dev;
  bs.form = tu.form;
  cudaError_t e;
  if (tu.form == 2) {
    // one graph node per depth of every array: k_gather_depth grids with no
    // dependencies between them, so that the GPU runs them side by side
    int max_smem = 0;
    for (int i = 0; i < n; ++i) {
      lfbp_plan p = plans[i];
      const std::vector<DepthTiling>& tl = plan_tiling(p, tu.tile_bytes);
      for (int z = 0; z < p->Nz; ++z) {
        if (p->off[z + 1] == p->off[z]) continue;
        const DepthTiling& dt = tl[z];
        DepthNode dn;
        dn.base = depth_desc(p, z, dt, (int)p->mode, i, tu.pairs);
        depth_shapes(p, z, dt, dn.base, dn.ds.s);
        dn.grid = dim3(dt.nV, p->Nx, dt.nU);
        dn.J = dt.J;
        dn.V = dt.V;
        dn.stage = (dt.max_tile_bytes + 15) & ~15;
        max_smem = std::max(max_smem, plain_smem_bytes(dn.stage));
        bs.ntiles += dt.nV * p->Nx * dt.nU;
        bs.dnodes.push_back(dn);
      }
    }
    if (max_smem > optin) return fail(LFBP_ERR_BAD_SHAPE, "tile does not fit in shared memory");
    if ((rc = ensure_smem_attr((const void*)k_gather_depth, max_smem))) return rc;
    if ((e = cudaGraphCreate(&bs.graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    std::memset(&bs.ptrs, 0, sizeof(bs.ptrs));
    bs.knodes.resize(bs.dnodes.size());
    for (size_t k = 0; k < bs.dnodes.size(); ++k) {
      DepthNodeArgs a;
      cudaKernelNodeParams kp;
      depth_node_params(bs, bs.dnodes[k], a, &kp);
      if ((e = cudaGraphAddKernelNode(&bs.knodes[k], bs.graph, nullptr, 0, &kp)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphAddKernelNode");
    }
    if (fault_mode() == kFaultGraph) return fail(LFBP_ERR_CUDA, "injected failure (LFBP_FAULT=graph)");
    if ((e = cudaGraphInstantiate(&bs.exec, bs.graph, 0)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphInstantiate");
    return LFBP_OK;
  }
  std::vector<TileDesc> tiles;
  std::vector<TileShape> shapes;
  int max_tile = 0;
  build_tiles(n, plans, tu.tile_bytes, tu.pairs, tiles, shapes, &max_tile);
  if (shapes.size() > 65536) return fail(LFBP_ERR_BAD_SHAPE, "more than 16384 depths in one batch");
  bs.ntiles = (int)tiles.size();
  bs.stage_bytes = (max_tile + 127) & ~127;
  if (tu.form == 1) {  // one tile per CTA: the whole list is the grid
    bs.nstages = 1;
    bs.smem = plain_smem_bytes(bs.stage_bytes);
    if (bs.smem > optin) return fail(LFBP_ERR_BAD_SHAPE, "tile does not fit in shared memory");
    bs.grid = std::max(1, bs.ntiles);
  } else {  // persistent CTAs: as many stages as fit next to the others on an SM
    const int cps = std::max(1, tu.ctas_per_sm);
    const int per_cta_budget = std::min(optin, (227 * 1024) / cps - 1024);
    const int per_stage = bs.stage_bytes + kInfoBytes + 16;  // as persistent_smem_bytes
    int nst = per_cta_budget / per_stage;
    if (tu.stages > 0) nst = std::min(nst, tu.stages);
    if (nst < 2) nst = std::min(2, optin / per_stage);
    if (nst < 1) return fail(LFBP_ERR_BAD_SHAPE, "tile does not fit in shared memory");
    bs.nstages = nst;
    bs.smem = persistent_smem_bytes(bs.stage_bytes, nst);
    bs.grid = std::max(1, std::min(sms * cps, bs.ntiles));
  }
  if (bs.ntiles) {
    if (fault_mode() == kFaultAlloc) return fail(LFBP_ERR_NOMEM, "injected failure (LFBP_FAULT=alloc)");
    const size_t tb = sizeof(TileDesc) * tiles.size(), sb = sizeof(TileShape) * shapes.size();
    if ((e = cudaMalloc(&bs.d_tiles, tb + sb)) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(tiles)");
    bs.d_shapes = reinterpret_cast<TileShape*>(reinterpret_cast<unsigned char*>(bs.d_tiles) + tb);
    if ((e = cudaMemcpy(bs.d_tiles, tiles.data(), tb, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy(tiles)");
    if ((e = cudaMemcpy(bs.d_shapes, shapes.data(), sb, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy(shapes)");
  }
  if ((rc = ensure_smem_attr(batch_fn(bs), bs.smem))) return rc;
  // a one-node graph: relaunching it costs one cudaGraphLaunch; pointer
  // changes are patched into the node's parameters
  if ((e = cudaGraphCreate(&bs.graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  std::memset(&bs.ptrs, 0, sizeof(bs.ptrs));
  void* args[6];
  cudaKernelNodeParams kp;
  batch_node_params(bs, args, &kp);
  if ((e = cudaGraphAddKernelNode(&bs.knode, bs.graph, nullptr, 0, &kp)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphAddKernelNode");
  if (fault_mode() == kFaultGraph) return fail(LFBP_ERR_CUDA, "injected failure (LFBP_FAULT=graph)");
  if ((e = cudaGraphInstantiate(&bs.exec, bs.graph, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphInstantiate");
  return LFBP_OK;
}

// Launches a built batch for the pointers np on st: patches the graph's
// node parameters when the pointers changed, then launches the graph.
int launch_batch(BatchState& bs, const BatchPtrs& np, cudaStream_t st) {
  cudaError_t e;
  if (std::memcmp(&np, &bs.ptrs, sizeof(np)) != 0) {
    bs.ptrs = np;
    if (bs.form == 2) {
      for (size_t k = 0; k < bs.dnodes.size(); ++k) {
        DepthNodeArgs a;
        cudaKernelNodeParams kp;
        depth_node_params(bs, bs.dnodes[k], a, &kp);
        if ((e = cudaGraphExecKernelNodeSetParams(bs.exec, bs.knodes[k], &kp)) != cudaSuccess)
          return cuda_fail(e, "cudaGraphExecKernelNodeSetParams");
      }
    } else {
      void* args[6];
      cudaKernelNodeParams kp;
      batch_node_params(bs, args, &kp);
      if ((e = cudaGraphExecKernelNodeSetParams(bs.exec, bs.knode, &kp)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphExecKernelNodeSetParams");
    }
  }
  if ((e = cudaGraphLaunch(bs.exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return LFBP_OK;
}

int run_batched(int n, const lfbp_plan* plans, const void* const* in, void* const* out,
                cudaStream_t st, int lsu_force) {
  const bool lsu = lsu_force >= 0 ? lsu_force != 0 : env_lsu();
  if (n < 0 || n > kMaxBatch) return fail(LFBP_ERR_INVALID, "batch size must be in [0, 64]");
  if (n == 0) return LFBP_OK;
  if (!plans || !in || !out) return fail(LFBP_ERR_NULL, "NULL array argument");
  for (int i = 0; i < n; ++i) {
    int rc = check_buffers(plans[i], in[i], out[i]);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const size_t bi = plans[i]->off.back() * plans[i]->es;
      const size_t bk = plans[k]->off.back() * plans[k]->es;
      if (bi && bk && overlaps(out[i], bi, in[k], bk))
        return fail(LFBP_ERR_ALIAS, "an output overlaps an input");
      if (k != i && bi && bk && overlaps(out[i], bi, out[k], bk))
        return fail(LFBP_ERR_ALIAS, "two outputs overlap");
    }
  if (batch_empty(n, plans)) return LFBP_OK;  // nothing to map: no CUDA call at all
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  Tuning want = tuning_for(dev, n, plans);
  if (fault_mode() == kFaultStall || lsu) want.form = 0;  // both need the persistent kernel
  BatchState* bs = nullptr;
  for (auto& b : g_batches) {
    if (b->dev != dev || b->lsu != lsu || !same_uids(b->uids, n, plans)) continue;
    if (b->tuning.tile_bytes != want.tile_bytes || b->tuning.ctas_per_sm != want.ctas_per_sm ||
        b->tuning.stages != want.stages || b->tuning.pairs != want.pairs ||
        b->tuning.form != want.form)
      continue;
    bs = b.get();
    break;
  }
  if (!bs) {
    if (g_batches.size() >= kMaxCachedBatches) {
      auto it = std::min_element(g_batches.begin(), g_batches.end(),
                                 [](const std::unique_ptr<BatchState>& a,
                                    const std::unique_ptr<BatchState>& b) {
                                   return a->last_use < b->last_use;
                                 });
      g_batches.erase(it);
    }
    std::unique_ptr<BatchState> nb(new BatchState());
    for (int i = 0; i < n; ++i) nb->uids.push_back(plans[i]->uid);
    nb->tuning = want;
    nb->lsu = lsu;
    int rc = build_batch(*nb, n, plans, want);
    if (rc) return rc;
    bs = nb.get();
    g_batches.push_back(std::move(nb));
  }
  bs->last_use = ++g_clock;
  if (bs->ntiles == 0) return LFBP_OK;
  BatchPtrs np;
  std::memset(&np, 0, sizeof(np));
  for (int i = 0; i < n; ++i) {
    np.in[i] = (const unsigned char*)in[i];
    np.out[i] = (unsigned char*)out[i];
    np.in_bytes[i] = plans[i]->off.back() * plans[i]->es;
  }
  if (fault_mode() == kFaultStall) {  // the injected kernel, launched directly
    bs->ptrs = np;
    int rc = ensure_smem_attr((const void*)k_gather_persistent<true>, bs->smem);
    if (rc) return rc;
    k_gather_persistent<true><<<bs->grid, kPersistentThreads, bs->smem, st>>>(
        bs->ptrs, bs->d_tiles, bs->d_shapes, bs->ntiles, bs->stage_bytes, bs->nstages);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_gather_persistent launch");
    return LFBP_OK;
  }
  return launch_batch(*bs, np, st);
}

// ------------------------------------------------------- no-allocation path --
// For callers that must not allocate device memory themselves or through this
// library (for instance code that owns a fixed memory pool, or a host
// framework that forbids cudaMalloc during its run), lfbp_backproject_batched_
// noalloc keeps the persistent kernel's work list in this file-scope device
// array instead of a cudaMalloc'd buffer.  Every GPU that loads the library
// holds the array until the process exits.
constexpr int kNoAllocMaxTiles = 262144;  // 8 MiB of 32-byte slots: tiles, then their shapes
static __device__ __align__(256) TileDesc g_noalloc_tiles[kNoAllocMaxTiles];
constexpr int kShapeSlots = (int)((sizeof(TileShape) + sizeof(TileDesc) - 1) / sizeof(TileDesc));

// Per device: the array's device address (from cudaGetSymbolAddress) and
// which work list it holds now.
struct NoAllocDev {
  int dev = -1;
  TileDesc* d_tiles = nullptr;
  int sms = 0, optin = 0;
  std::vector<unsigned long long> uids;  // plans of the list in the array
  TileShape* d_shapes = nullptr;  // inside the array, after the tiles
  int tile_bytes = 0, ntiles = 0, stage_bytes = 0, nstages = 0, grid = 0, smem = 0;
};
std::vector<std::unique_ptr<NoAllocDev>> g_noalloc;  // guarded by g_mu

// Set-up, once per device, with that device current: the host-side name of
// the array is not a device address, so ask the runtime for it.
int noalloc_setup(int dev, NoAllocDev** out) {
  for (auto& d : g_noalloc)
    if (d->dev == dev) {
      *out = d.get();
      return LFBP_OK;
    }
  std::unique_ptr<NoAllocDev> nd(new NoAllocDev());
  nd->dev = dev;
  cudaError_t e = cudaGetSymbolAddress((void**)&nd->d_tiles, g_noalloc_tiles);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(work list array)");
  int d2 = 0;
  int rc = device_props(&d2, &nd->sms, &nd->optin);
  if (rc) return rc;
  *out = nd.get();
  g_noalloc.push_back(std::move(nd));
  return LFBP_OK;
}

// Tile-size target and tile count of a batch on the no-allocation path: the
// default target, or larger tiles (fewer descriptors) when the list would not
// fit the array.  Host only: no CUDA call.
void noalloc_target(int n, const lfbp_plan* plans, const Tuning& dflt, int* target,
                    long long* need) {
  *target = dflt.tile_bytes;
  for (int t : {dflt.tile_bytes, std::max(dflt.tile_bytes, 49152)}) {
    *target = t;
    *need = 0;
    for (int i = 0; i < n; ++i) {
      const std::vector<DepthTiling>& tl = plan_tiling(plans[i], t);
      for (int z = 0; z < plans[i]->Nz; ++z)
        *need += (long long)plans[i]->Nx * tl[z].nU * tl[z].nV + 4 * kShapeSlots;  // tiles + shapes
    }
    if (*need <= kNoAllocMaxTiles) return;
  }
}

int run_batched_noalloc(int n, const lfbp_plan* plans, const void* const* in, void* const* out,
                        cudaStream_t st) {
  if (n < 0 || n > kMaxBatch) return fail(LFBP_ERR_INVALID, "batch size must be in [0, 64]");
  if (n == 0) return LFBP_OK;
  if (!plans || !in || !out) return fail(LFBP_ERR_NULL, "NULL array argument");
  for (int i = 0; i < n; ++i) {
    int rc = check_buffers(plans[i], in[i], out[i]);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const size_t bi = plans[i]->off.back() * plans[i]->es;
      const size_t bk = plans[k]->off.back() * plans[k]->es;
      if (bi && bk && overlaps(out[i], bi, in[k], bk))
        return fail(LFBP_ERR_ALIAS, "an output overlaps an input");
      if (k != i && bi && bk && overlaps(out[i], bi, out[k], bk))
        return fail(LFBP_ERR_ALIAS, "two outputs overlap");
    }
  if (batch_empty(n, plans)) return LFBP_OK;  // nothing to map: no CUDA call at all
  // the size check comes before any CUDA call, so a batch too large for the
  // array is refused without touching the device or the buffers
  // the persistent kernel, in its own default shape (32 KB tiles unless set)
  Tuning tu = default_tuning();
  tu.form = 0;
  tu.tile_bytes = std::min(65536, std::max(1024, env_int("LFBP_TILE_BYTES", 32768)));
  long long need = 0;
  noalloc_target(n, plans, tu, &tu.tile_bytes, &need);
  if (need > kNoAllocMaxTiles) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "the batch needs %lld descriptor slots (tiles and tile shapes); the "
                  "no-allocation path holds at most %d",
                  need, kNoAllocMaxTiles);
    return fail(LFBP_ERR_BAD_SHAPE, msg);
  }
  if (need == 0) return LFBP_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDev* nd = nullptr;
  int rc = noalloc_setup(dev, &nd);
  if (rc) return rc;
  bool loaded = nd->tile_bytes == tu.tile_bytes && same_uids(nd->uids, n, plans);
  if (!loaded) {
    // the new list is copied from host memory owned by this call; such a copy
    // cannot be ordered into a stream that is being captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
      return fail(LFBP_ERR_INVALID,
                  "the work list must be replaced, which cannot be done while the stream is "
                  "capturing");
    std::vector<TileDesc> tiles;
    std::vector<TileShape> shapes;
    tiles.reserve((size_t)need);
    int max_tile = 0;
    build_tiles(n, plans, tu.tile_bytes, tu.pairs, tiles, shapes, &max_tile);
    const int stage_bytes = (max_tile + 127) & ~127;
    const int per_cta_budget = std::min(nd->optin, (227 * 1024) / tu.ctas_per_sm - 1024);
    const int per_stage = stage_bytes + kInfoBytes + 16;  // as persistent_smem_bytes
    int nst = per_cta_budget / per_stage;
    if (tu.stages > 0) nst = std::min(nst, tu.stages);
    if (nst < 2) nst = std::min(2, nd->optin / per_stage);
    if (nst < 1) return fail(LFBP_ERR_BAD_SHAPE, "tile does not fit in shared memory");
    // stream-ordered: the kernels of earlier calls on this stream have read
    // the previous list before this copy overwrites it
    TileShape* d_shapes = reinterpret_cast<TileShape*>(nd->d_tiles + tiles.size());
    if ((e = cudaMemcpyAsync(nd->d_tiles, tiles.data(), sizeof(TileDesc) * tiles.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(work list)");
    if ((e = cudaMemcpyAsync(d_shapes, shapes.data(), sizeof(TileShape) * shapes.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync(tile shapes)");
    nd->d_shapes = d_shapes;
    // the copy reads `tiles` (pageable host memory) before returning
    nd->uids.clear();
    for (int i = 0; i < n; ++i) nd->uids.push_back(plans[i]->uid);
    nd->tile_bytes = tu.tile_bytes;
    nd->ntiles = (int)tiles.size();
    nd->stage_bytes = stage_bytes;
    nd->nstages = nst;
    nd->smem = persistent_smem_bytes(stage_bytes, nst);
    nd->grid = std::max(1, std::min(nd->sms * tu.ctas_per_sm, nd->ntiles));
  }
  if ((rc = ensure_smem_attr((const void*)k_gather_persistent<false>, nd->smem))) return rc;
  BatchPtrs np;
  std::memset(&np, 0, sizeof(np));
  for (int i = 0; i < n; ++i) {
    np.in[i] = (const unsigned char*)in[i];
    np.out[i] = (unsigned char*)out[i];
    np.in_bytes[i] = plans[i]->off.back() * plans[i]->es;
  }
  if (fault_mode() == kFaultStall) {
    if ((rc = ensure_smem_attr((const void*)k_gather_persistent<true>, nd->smem))) return rc;
    k_gather_persistent<true><<<nd->grid, kPersistentThreads, nd->smem, st>>>(
        np, nd->d_tiles, nd->d_shapes, nd->ntiles, nd->stage_bytes, nd->nstages);
  } else {
    k_gather_persistent<false><<<nd->grid, kPersistentThreads, nd->smem, st>>>(
        np, nd->d_tiles, nd->d_shapes, nd->ntiles, nd->stage_bytes, nd->nstages);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_gather_persistent launch");
  return LFBP_OK;
}

// ------------------------------------------------------------------ tuner --
// Shape signature of a list of plans (for the tuning cache file).
std::string plans_signature(int dev, int n, const lfbp_plan* plans) {
  cudaDeviceProp prop;
  std::string sig;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) sig += prop.name;
  for (int i = 0; i < n; ++i) {
    lfbp_plan p = plans[i];
    char buf[96];
    std::snprintf(buf, sizeof(buf), "|%d:%d:%d:%d:%d", p->Nx, p->Ny, p->es, (int)p->mode, p->Nz);
    sig += buf;
    unsigned long long h = 1469598103934665603ull;
    for (int z = 0; z < p->Nz; ++z) {
      h = (h ^ (unsigned long long)p->Ks[z]) * 1099511628211ull;
      h = (h ^ (unsigned long long)p->Kt[z]) * 1099511628211ull;
    }
    std::snprintf(buf, sizeof(buf), ":%016llx", h);
    sig += buf;
  }
  for (char& ch : sig)
    if (ch == ' ' || ch == '\n' || ch == '\t') ch = '_';
  return sig;
}

bool cache_lookup(const std::string& sig, Tuning* t) {
  const char* path = std::getenv("LFBP_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char key[4096];
  Tuning x{0, 0, 0, 1, 0};
  bool found = false;
  while (std::fscanf(f, "%4095s %d %d %d %d %d", key, &x.tile_bytes, &x.ctas_per_sm, &x.stages,
                     &x.pairs, &x.form) == 6)
    if (sig == key) {
      *t = x;
      found = true;
    }
  std::fclose(f);
  return found;
}

void cache_store(const std::string& sig, const Tuning& t) {
  const char* path = std::getenv("LFBP_TUNE_CACHE");
  if (!path || !*path || sig.size() > 4000) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %d\n", sig.c_str(), t.tile_bytes, t.ctas_per_sm, t.stages,
               t.pairs, t.form);
  std::fclose(f);
}

int tune_batched(int n, const lfbp_plan* plans, const void* const* in, void* const* out,
                 cudaStream_t st, int reps, Tuning* chosen) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const bool lsu = env_lsu();
  const std::string sig = plans_signature(dev, n, plans) + (lsu ? "/lsu" : "");
  Tuning best = default_tuning();
  if (!cache_lookup(sig, &best)) {
    const int tiles[] = {12288, 16384, 24576, 32768, 40960, 49152, 65536};
    const int ctas[] = {1, 2, 3, 4};
    float best_ms = 1e30f;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&b)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    BatchPtrs np;
    std::memset(&np, 0, sizeof(np));
    for (int i = 0; i < n; ++i) {
      np.in[i] = (const unsigned char*)in[i];
      np.out[i] = (unsigned char*)out[i];
      np.in_bytes[i] = plans[i]->off.back() * plans[i]->es;
    }
    int rc = LFBP_OK;
    // the candidates: persistent CTAs (tile size x CTAs per SM) and one tile
    // per CTA (tile size), each with the pair consumer on and off
    std::vector<Tuning> cands;
    for (int pr = 1; pr >= 0; --pr) {
      for (int tb : tiles)
        for (int cp : ctas) cands.push_back(Tuning{tb, cp, 0, pr, 0});
      if (!lsu)
        for (int tb : tiles)
          if (tb >= 24576)
            for (int form = 1; form <= 2; ++form) cands.push_back(Tuning{tb, 0, 0, pr, form});
    }
    for (const Tuning& t : cands) {
        BatchState bs;
        bs.lsu = lsu;
        if (build_batch(bs, n, plans, t) != LFBP_OK || (t.form == 0 && bs.nstages < 2)) {
          cudaGetLastError();
          continue;
        }
        if (bs.ntiles == 0) continue;
        for (int r = 0; r <= reps; ++r) {
          if (r == 1) cudaEventRecord(a, st);
          if ((rc = launch_batch(bs, np, st)) != LFBP_OK) break;
        }
        if (rc) break;
        cudaEventRecord(b, st);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
          rc = cuda_fail(e, "tuning launch");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= (float)(reps > 0 ? reps : 1);
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    cache_store(sig, best);
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    bool done = false;
    for (TunedEntry& t : g_tuned)
      if (t.dev == dev && same_uids(t.uids, n, plans)) {
        t.tuning = best;
        done = true;
      }
    if (!done) {
      TunedEntry te;
      te.dev = dev;
      for (int i = 0; i < n; ++i) te.uids.push_back(plans[i]->uid);
      te.tuning = best;
      g_tuned.push_back(te);
    }
  }
  if (chosen) *chosen = best;
  return LFBP_OK;
}

// `a`: the plan-sized array (H or H'), or with a_bytes > 0 an input of that
// many bytes; `out`: the output, out_bytes long.
int check_projector(lfbp_plan p, const void* a, const void* b, const void* out, int Wx, int Wy,
                    size_t out_bytes, size_t a_bytes = 0) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  if (p->dt != LFBP_F32) return fail(LFBP_ERR_DTYPE, "projectors need an LFBP_F32 plan");
  if (Wx < 1 || Wy < 1) return fail(LFBP_ERR_BAD_SHAPE, "sensor must be at least 1 x 1");
  for (int z = 0; z < p->Nz; ++z)
    if (p->Kt[z] > 3072) return fail(LFBP_ERR_BAD_SHAPE, "projectors need Kt <= 3072");
  if (p->literal) return fail(LFBP_ERR_BAD_SHAPE, "projectors need odd cut-outs");
  if ((p->Nz > 0 && !a) || !b || !out) return fail(LFBP_ERR_NULL, "buffer pointer is NULL");
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)out) & 3)
    return fail(LFBP_ERR_ALIGN, "buffers must be 4-byte aligned");
  const size_t sa = a_bytes ? a_bytes : p->off.back() * 4;
  if (a && overlaps(a, sa, out, out_bytes)) return fail(LFBP_ERR_ALIAS, "output overlaps an input");
  return LFBP_OK;
}

int make_plan(lfbp_plan* out, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
              lfbp_dtype dt, lfbp_mode mode) {
  if (!out) return fail(LFBP_ERR_NULL, "out is NULL");
  *out = nullptr;
  if (fault_mode() == kFaultPlan) return fail(LFBP_ERR_NOMEM, "injected failure (LFBP_FAULT=plan)");
  if (Nz < 0) return fail(LFBP_ERR_BAD_SHAPE, "Nz must be >= 0");
  if (Nz > 0 && (!Ks || !Kt)) return fail(LFBP_ERR_NULL, "Ks/Kt is NULL");
  if (Nx < 1 || Ny < 1 || Nx % 2 == 0 || Ny % 2 == 0)
    return fail(LFBP_ERR_BAD_SHAPE, "Nx and Ny must be odd and >= 1");
  if (Nx > 1023 || Ny > 1023) return fail(LFBP_ERR_BAD_SHAPE, "Nx and Ny must be <= 1023");
  if (dt != LFBP_F32 && dt != LFBP_F16) return fail(LFBP_ERR_DTYPE, "unknown dtype");
  if (mode != LFBP_MAP_TRANSPOSE && mode != LFBP_MAP_PAPER_WINDOW)
    return fail(LFBP_ERR_INVALID, "unknown mode");
  std::unique_ptr<lfbp_plan_s> p(new lfbp_plan_s());
  p->Nx = Nx;
  p->Ny = Ny;
  p->Nz = Nz;
  p->dt = dt;
  p->mode = mode;
  p->es = dt == LFBP_F32 ? 4 : 2;
  p->off.push_back(0);
  for (int z = 0; z < Nz; ++z) {
    const int ks = Ks[z], kt = Kt[z];
    if (ks < 1 || kt < 1) return fail(LFBP_ERR_BAD_SHAPE, "every Ks and Kt must be >= 1");
    if (ks % 2 == 0 || kt % 2 == 0) {
      // Eq. 8 with even n_s is a partial map (reading A2): only the literal
      // paper window defines it
      if (mode != LFBP_MAP_PAPER_WINDOW)
        return fail(LFBP_ERR_BAD_SHAPE,
                    "even Ks or Kt: the transpose needs odd cut-outs (use LFBP_MAP_PAPER_WINDOW "
                    "for the literal Eq. 8)");
      p->literal = true;
    }
    if (ks > 16383 || kt > 16383) return fail(LFBP_ERR_BAD_SHAPE, "Ks and Kt must be <= 16383");
    p->Ks.push_back(ks);
    p->Kt.push_back(kt);
    p->off.push_back(p->off.back() + (size_t)Nx * Ny * (size_t)ks * kt);
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    p->uid = g_next_uid++;
  }
  *out = p.release();
  return LFBP_OK;
}

}  // namespace

// ===================================================================== C-ABI
extern "C" {

int lfbp_plan_create(lfbp_plan* out, int Nnum, int Nz, const int* Kz, lfbp_dtype dt,
                     lfbp_mode mode) {
  return make_plan(out, Nnum, Nnum, Nz, Kz, Kz, dt, mode);
}

int lfbp_plan_create2(lfbp_plan* out, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
                      lfbp_dtype dt, lfbp_mode mode) {
  return make_plan(out, Nx, Ny, Nz, Ks, Kt, dt, mode);
}

void lfbp_plan_destroy(lfbp_plan p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_tuned.size();) {
      bool uses = false;
      for (auto u : g_tuned[i].uids) uses |= (u == p->uid);
      if (uses)
        g_tuned.erase(g_tuned.begin() + i);
      else
        ++i;
    }
    for (size_t i = 0; i < g_batches.size();) {
      bool uses = false;
      for (auto u : g_batches[i]->uids) uses |= (u == p->uid);
      if (uses)
        g_batches.erase(g_batches.begin() + i);
      else
        ++i;
    }
  }
  delete p;
}

size_t lfbp_plan_elems(lfbp_plan p) { return p ? p->off.back() : 0; }

size_t lfbp_plan_depth_offset(lfbp_plan p, int z) {
  if (!p || z < 0 || z > p->Nz) return 0;
  return p->off[z];
}

int lfbp_plan_esize(lfbp_plan p) { return p ? p->es : 0; }

int lfbp_plan_partition(lfbp_plan p, int nparts, int part, int* z0, int* z1) {
  if (!p || !z0 || !z1) return fail(LFBP_ERR_NULL, "NULL argument");
  if (nparts < 1 || part < 0 || part >= nparts) return fail(LFBP_ERR_INVALID, "part out of range");
  // boundary k sits at the depth start nearest to k/nparts of the elements
  // (non-decreasing in k: the targets grow and ties keep the first depth); the
  // depths are independent (Sec. 4), so a part is any contiguous range
  const double total = (double)p->off.back();
  auto boundary = [&](int k) {
    if (k <= 0) return 0;
    if (k >= nparts) return p->Nz;
    const double target = total * k / nparts;
    int best = 0;
    for (int z = 1; z <= p->Nz; ++z)
      if (std::fabs((double)p->off[z] - target) < std::fabs((double)p->off[best] - target)) best = z;
    return best;
  };
  *z0 = boundary(part);
  *z1 = std::max(*z0, boundary(part + 1));
  return LFBP_OK;
}

int lfbp_backproject_array(lfbp_plan p, const void* dH, void* dHp, void* cuda_stream) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  return run_plain(p, dH, dHp, (int)p->mode, (cudaStream_t)cuda_stream);
}

int lfbp_backproject_array_host(lfbp_plan p, const void* H_host, void* Hp_host, void* dH_work,
                                void* dHp_work, void* cuda_stream) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  return run_host(p, H_host, Hp_host, dH_work, dHp_work, (int)p->mode, (cudaStream_t)cuda_stream);
}

int lfbp_backproject_batched(int n, const lfbp_plan* plans, const void* const* dH,
                             void* const* dHp, void* cuda_stream) {
  return run_batched(n, plans, dH, dHp, (cudaStream_t)cuda_stream, -1);
}

int lfbp_backproject_batched_noalloc(int n, const lfbp_plan* plans, const void* const* dH,
                                     void* const* dHp, void* cuda_stream) {
  return run_batched_noalloc(n, plans, dH, dHp, (cudaStream_t)cuda_stream);
}

int lfbp_tune_batched(int n, const lfbp_plan* plans, const void* const* dH, void* const* dHp,
                      void* cuda_stream, int reps, int* tuned) {
  int rc = run_batched(n, plans, dH, dHp, (cudaStream_t)cuda_stream, -1);  // validates the arguments
  if (rc) return rc;
  if (n == 0) return LFBP_OK;
  Tuning t{0, 0, 0, 0, 0};
  rc = tune_batched(n, plans, dH, dHp, (cudaStream_t)cuda_stream, reps < 1 ? 3 : reps, &t);
  if (rc) return rc;
  if (tuned) {
    tuned[0] = t.tile_bytes;
    tuned[1] = t.ctas_per_sm;
    tuned[2] = t.stages;
    tuned[3] = t.pairs;
    tuned[4] = t.form;
  }
  return LFBP_OK;
}

int lfbp_adjoint(lfbp_plan p, const void* dHp_grad, void* dH_grad, void* cuda_stream) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  const int mode = p->mode == LFBP_MAP_TRANSPOSE ? 0 : 2;
  return run_plain(p, dHp_grad, dH_grad, mode, (cudaStream_t)cuda_stream);
}

namespace {

// A projection over all depths of the plan as output-cell sums (see
// lfbp_project.h): `mapped` reads the weights through the map of A.  Depths
// whose cut-out exceeds the phase kernel's sizes take the direct kernel,
// which reads the unmapped array `A_direct` with source-cell patterns.
int project(lfbp_plan p, const float* A, int mapped, const float* A_direct, int direct_out_cell,
            const float* in, long long in_zs, float* out, long long out_zs, const float* g,
            const float* norm, int Wx, int Wy, int sum_depths, int epi, cudaStream_t st) {
  std::vector<long long> off(p->Nz);
  for (int z = 0; z < p->Nz; ++z) off[z] = (long long)p->off[z];
  int* status = nullptr;
  if (cudaGetSymbolAddress((void**)&status, g_status) != cudaSuccess)
    return fail(LFBP_ERR_CUDA, "cudaGetSymbolAddress(status)");
  const int rc = launch_phase_projection(A, mapped, p->Nx, p->Ny, p->Nz, off.data(), p->Ks.data(),
                                         p->Kt.data(), in, in_zs, out, out_zs, g, norm, Wx, Wy,
                                         sum_depths, epi, status, st);
  if (rc == 0) return LFBP_OK;
  if (rc != -1) return fail(LFBP_ERR_CUDA, "k_phase_conv launch failed");
  for (int z = 0; z < p->Nz; ++z) {
    const int e = sum_depths ? (z ? kEpiAccumulate : epi) : epi;
    const long long o = sum_depths ? 0 : (long long)z * out_zs;
    if (launch_projector(direct_out_cell, e, A_direct + p->off[z], p->Nx, p->Ny, p->Ks[z],
                         p->Kt[z], in + (long long)z * in_zs, Wx, Wy, out + o, g ? g + o : nullptr,
                         norm ? norm + o : nullptr, st))
      return fail(LFBP_ERR_CUDA, "k_shift_variant_sum launch failed");
  }
  return LFBP_OK;
}

}  // namespace

int lfbp_backproject_volume(lfbp_plan p, const void* dHp, const float* df, int Wx, int Wy,
                            float* dg, void* cuda_stream) {
  int rc = check_projector(p, dHp, df, dg, Wx, Wy, (size_t)(p ? p->Nz : 0) * Wx * Wy * 4);
  if (rc) return rc;
  if (overlaps(df, (size_t)Wx * Wy * 4, dg, (size_t)p->Nz * Wx * Wy * 4))
    return fail(LFBP_ERR_ALIAS, "output overlaps an input");
  const float* hp = (const float*)dHp;
  // weights H[p][q] = the map of H' (its own inverse)
  return project(p, hp, 1, hp, 0, df, 0, dg, (long long)Wx * Wy, nullptr, nullptr, Wx, Wy, 0,
                 kEpiStore, (cudaStream_t)cuda_stream);
}

int lfbp_forward_project(lfbp_plan p, const void* dH, const float* dg, int Wx, int Wy, float* df,
                         void* cuda_stream) {
  int rc = check_projector(p, dH, dg, df, Wx, Wy, (size_t)Wx * Wy * 4);
  if (rc) return rc;
  if (overlaps(df, (size_t)Wx * Wy * 4, dg, (size_t)p->Nz * Wx * Wy * 4))
    return fail(LFBP_ERR_ALIAS, "output overlaps an input");
  const float* h = (const float*)dH;
  if (p->Nz == 0) {
    cudaError_t e = cudaMemsetAsync(df, 0, (size_t)Wx * Wy * 4, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    return LFBP_OK;
  }
  // weights H'[p][q] = the map of H; depths summed in order
  return project(p, h, 1, h, 0, dg, (long long)Wx * Wy, df, 0, nullptr, nullptr, Wx, Wy, 1,
                 kEpiStore, (cudaStream_t)cuda_stream);
}

int lfbp_backproject_volume_grad(lfbp_plan p, const float* df, const float* dgrad, int Wx, int Wy,
                                 void* dHp_grad, void* cuda_stream) {
  // dgrad is the Nz x Wx x Wy gradient volume, not a plan-sized array
  int rc = check_projector(p, dgrad, df, dHp_grad, Wx, Wy, p ? p->off.back() * 4 : 0,
                           (size_t)(p ? p->Nz : 0) * Wx * Wy * 4);
  if (rc) return rc;
  if (overlaps(df, (size_t)Wx * Wy * 4, dHp_grad, p->off.back() * 4))
    return fail(LFBP_ERR_ALIAS, "output overlaps an input");
  float* out = (float*)dHp_grad;
  std::vector<long long> off(p->Nz);
  for (int z = 0; z < p->Nz; ++z) off[z] = (long long)p->off[z];
  int* status = nullptr;
  if (cudaGetSymbolAddress((void**)&status, g_status) != cudaSuccess)
    return fail(LFBP_ERR_CUDA, "cudaGetSymbolAddress(status)");
  const int prc = launch_phase_grad(df, dgrad, p->Nx, p->Ny, p->Nz, off.data(), p->Ks.data(),
                                    p->Kt.data(), Wx, Wy, out, status, (cudaStream_t)cuda_stream);
  if (prc == 0) return LFBP_OK;
  if (prc != -1) return fail(LFBP_ERR_CUDA, "k_phase_grad launch failed");
  for (int z = 0; z < p->Nz; ++z) {
    if (launch_backproject_grad(df, dgrad + (size_t)z * Wx * Wy, p->Nx, p->Ny, p->Ks[z], p->Kt[z],
                                Wx, Wy, out + p->off[z], (cudaStream_t)cuda_stream))
      return fail(LFBP_ERR_CUDA, "k_backproject_grad launch failed");
  }
  return LFBP_OK;
}

int lfbp_backproject_volume_from_h(lfbp_plan p, const void* dH, const float* df, int Wx, int Wy,
                                   float* dg, void* cuda_stream) {
  int rc = check_projector(p, dH, df, dg, Wx, Wy, (size_t)(p ? p->Nz : 0) * Wx * Wy * 4);
  if (rc) return rc;
  if (overlaps(df, (size_t)Wx * Wy * 4, dg, (size_t)p->Nz * Wx * Wy * 4))
    return fail(LFBP_ERR_ALIAS, "output overlaps an input");
  const float* h = (const float*)dH;
  return project(p, h, 0, h, 1, df, 0, dg, (long long)Wx * Wy, nullptr, nullptr, Wx, Wy, 0,
                 kEpiStore, (cudaStream_t)cuda_stream);
}

namespace {

bool misaligned4(const void* a) { return ((uintptr_t)a & 3) != 0; }

// One Richardson-Lucy update (Eq. 2); dHp == nullptr: backprojection from H.
int rl_step_impl(lfbp_plan p, const void* dH, const void* dHp, const float* dnorm,
                 const float* df, int Wx, int Wy, const float* dg, float* dg_next, float* dwork,
                 cudaStream_t st) {
  int rc = check_projector(p, dH, df, dwork, Wx, Wy, (size_t)Wx * Wy * 4);
  if (rc) return rc;
  if (!dnorm || !dg || !dg_next) return fail(LFBP_ERR_NULL, "buffer pointer is NULL");
  if (misaligned4(dnorm) || misaligned4(dg) || misaligned4(dg_next) || misaligned4(dHp))
    return fail(LFBP_ERR_ALIGN, "buffers must be 4-byte aligned");
  const size_t img = (size_t)Wx * Wy * 4, vol = (size_t)p->Nz * img, hb = p->off.back() * 4;
  // the scratch image overlaps nothing; the new estimate overlaps nothing but
  // (exactly) the old one
  const void* reads[] = {df, dnorm, dg, dHp};
  const size_t rbytes[] = {img, vol, vol, hb};
  for (int i = 0; i < 4; ++i)
    if (reads[i] && overlaps(reads[i], rbytes[i], dwork, img))
      return fail(LFBP_ERR_ALIAS, "dwork overlaps another buffer");
  if (overlaps(dwork, img, dg_next, vol)) return fail(LFBP_ERR_ALIAS, "dwork overlaps dg_next");
  if (overlaps(dH, hb, dg_next, vol) || (dHp && overlaps(dHp, hb, dg_next, vol)) ||
      overlaps(dnorm, vol, dg_next, vol) || overlaps(df, img, dg_next, vol))
    return fail(LFBP_ERR_ALIAS, "dg_next overlaps an input");
  if ((const void*)dg != (const void*)dg_next && overlaps(dg, vol, dg_next, vol))
    return fail(LFBP_ERR_ALIAS, "dg_next overlaps dg without being dg");
  const float* h = (const float*)dH;
  const float* hp = (const float*)dHp;
  const long long W2 = (long long)Wx * Wy;
  if (p->Nz == 0) {
    cudaError_t e = cudaMemsetAsync(dwork, 0, img, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (launch_rl_quotient(df, dwork, W2, st))
      return fail(LFBP_ERR_CUDA, "k_rl_quotient launch failed");
  } else if ((const void*)dg_next != (const void*)dg) {
    // H g as per-depth partials in dg_next (one block per depth and tile: the
    // whole GPU busy), then their fixed-order sum and the quotient f / (H g)
    // into dwork; the update below overwrites the partials after their use
    rc = hp ? project(p, hp, 0, h, 0, dg, W2, dg_next, W2, nullptr, nullptr, Wx, Wy, 0, kEpiStore, st)
            : project(p, h, 1, h, 0, dg, W2, dg_next, W2, nullptr, nullptr, Wx, Wy, 0, kEpiStore, st);
    if (rc) return rc;
    if (launch_rl_sum_quotient(dg_next, p->Nz, W2, df, dwork, st))
      return fail(LFBP_ERR_CUDA, "k_rl_sum_quotient launch failed");
  } else {
    // in place: H g summed over depths inside each block, then f / (H g)
    rc = hp ? project(p, hp, 0, h, 0, dg, W2, dwork, 0, nullptr, nullptr, Wx, Wy, 1, kEpiStore, st)
            : project(p, h, 1, h, 0, dg, W2, dwork, 0, nullptr, nullptr, Wx, Wy, 1, kEpiStore, st);
    if (rc) return rc;
    if (launch_rl_quotient(df, dwork, W2, st))
      return fail(LFBP_ERR_CUDA, "k_rl_quotient launch failed");
  }
  // g / (H'1) * H' (f / (H g)), depth by depth (weights: H, or the map of H')
  return hp ? project(p, hp, 1, hp, 0, dwork, 0, dg_next, W2, dg, dnorm, Wx, Wy, 0, kEpiRL, st)
            : project(p, h, 0, h, 1, dwork, 0, dg_next, W2, dg, dnorm, Wx, Wy, 0, kEpiRL, st);
}

}  // namespace

int lfbp_rl_step(lfbp_plan p, const void* dH, const void* dHp, const float* dnorm,
                 const float* df, int Wx, int Wy, const float* dg, float* dg_next, float* dwork,
                 void* cuda_stream) {
  if (!dHp) return fail(LFBP_ERR_NULL, "dHp is NULL (lfbp_rl_step_fused needs no H')");
  return rl_step_impl(p, dH, dHp, dnorm, df, Wx, Wy, dg, dg_next, dwork,
                      (cudaStream_t)cuda_stream);
}

int lfbp_rl_step_fused(lfbp_plan p, const void* dH, const float* dnorm, const float* df, int Wx,
                       int Wy, const float* dg, float* dg_next, float* dwork, void* cuda_stream) {
  return rl_step_impl(p, dH, nullptr, dnorm, df, Wx, Wy, dg, dg_next, dwork,
                      (cudaStream_t)cuda_stream);
}

int lfbp_rl_normaliser(lfbp_plan p, const void* dH, const void* dHp, int Wx, int Wy, float* dnorm,
                       float* dwork, void* cuda_stream) {
  const void* A = dHp ? dHp : dH;
  int rc = check_projector(p, A, dwork, dnorm, Wx, Wy, (size_t)(p ? p->Nz : 0) * Wx * Wy * 4);
  if (rc) return rc;
  const size_t img = (size_t)Wx * Wy * 4;
  if (overlaps(dwork, img, dnorm, (size_t)p->Nz * img))
    return fail(LFBP_ERR_ALIAS, "dwork overlaps dnorm");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (launch_fill(dwork, (long long)Wx * Wy, 1.0f, st))
    return fail(LFBP_ERR_CUDA, "k_fill launch failed");
  const float* a = (const float*)A;
  return project(p, a, dHp ? 1 : 0, a, dHp ? 0 : 1, dwork, 0, dnorm, (long long)Wx * Wy, nullptr,
                 nullptr, Wx, Wy, 0, kEpiStore, st);
}

int lfbp_sync_status(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
#if LFBP_CHECKED
  {
    CheckWord cw;
    if ((e = cudaMemcpyFromSymbol(&cw, g_check, sizeof(cw))) != cudaSuccess)
      return cuda_fail(e, "read check word");
    if (cw.code != 0) {
      CheckWord zero;
      std::memset(&zero, 0, sizeof(zero));
      cudaMemcpyToSymbol(g_check, &zero, sizeof(zero));
      char msg[256];
      std::snprintf(msg, sizeof(msg),
                    "self-check violation: code %d (1 smem load, 2 store, 3 bulk copy, 4 tail "
                    "load) block %d thread %d values %lld %lld",
                    cw.code, cw.block, cw.thread, cw.a, cw.b);
      return fail(LFBP_ERR_INVALID, msg);
    }
  }
#endif
  int v = 0;
  if ((e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "read status");
  if (v != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
    return fail(v, v == LFBP_ERR_TIMEOUT ? "an in-kernel wait timed out; output incomplete"
                                         : "a kernel was launched with too little shared memory");
  }
  return LFBP_OK;
}

const char* lfbp_last_error(void) { return t_err.c_str(); }

const char* lfbp_version(void) {
#if LFBP_CHECKED
  return "lfbp 0.1 (sm_103a, self-checking build)";
#else
  return "lfbp 0.1 (sm_103a)";
#endif
}

}  // extern "C"
