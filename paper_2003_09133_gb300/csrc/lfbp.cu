// lfbp: H -> H' backprojection-array construction on one GPU (sm_103a).
//
// Kernels (see lfbp_device.cuh for the tile and the index map):
//   k_gather_depth       one tile per CTA, one launch per depth (the plain form)
//   k_gather_persistent  persistent CTAs over a ragged work list of all depths
//                        of all arrays; one producer warp streams tiles into a
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

namespace lfbp {

// Status word of the library on each device: 0 or a negative LFBP_ERR_* code
// written by a kernel whose bounded wait gave up.
__device__ int g_status;

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per in-kernel wait
constexpr int kPlainThreads = 256;
constexpr int kConsumerWarps = 8;
constexpr int kPersistentThreads = 32 * (1 + kConsumerWarps);
constexpr int kInfoBytes = 256;  // per-stage TileInfo slot (aligned)
static_assert(sizeof(TileInfo) <= kInfoBytes, "TileInfo too large");

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status, 0, code); }

// ------------------------------------------------------------------ plain --
// grid = (nV, Nx, nU) tiles of one depth; block = kPlainThreads.
// smem: [stage: tile bytes][TileInfo][mbarrier]
__global__ void __launch_bounds__(kPlainThreads)
    k_gather_depth(JobDesc jd, const unsigned char* __restrict__ in_depth,
                   const unsigned char* in_safe_end, unsigned char* __restrict__ out_depth, int J,
                   int V, int stage_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stage = smem;
  TileInfo* ti = reinterpret_cast<TileInfo*>(smem + stage_bytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + stage_bytes + kInfoBytes);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  TileDesc td;
  td.job = 0;
  td.p = (unsigned short)blockIdx.y;
  const int u0 = blockIdx.z * J, v0 = blockIdx.x * V;
  td.u0 = (unsigned short)u0;
  td.v0 = (unsigned short)v0;
  td.nrows = (unsigned short)min(J, jd.Ks - u0);
  td.ncols = (unsigned short)min(V, jd.Kt - v0);
  td.pad = 0;

  const uint32_t b = smem_addr(bar);
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(b, 1);
    fence_mbar_init();
    make_tile_info(*ti, 0, td, jd, in_depth, out_depth);
  }
  __syncthreads();
  if (warp == 0) issue_tile_loads(td, jd, in_depth, in_safe_end, stage, b, lane);
  if (!mbar_wait_bounded(b, 0, &abort_flag, kWaitLimitNs)) {
    set_status(kStatusTimeout);
    abort_flag = 1;
    // give the copies in flight a last bounded chance to land before exit
    mbar_wait_bounded(b, 0, nullptr, kWaitLimitNs);
    return;
  }
  gather_store_dispatch(*ti, stage, tid, kPlainThreads);
}

// ------------------------------------------------------------- persistent --
// grid = SMs * ctas_per_sm; block = kPersistentThreads.
// smem: [nstages x stage_bytes][nstages x TileInfo][full[nstages]][empty[nstages]]
__global__ void __launch_bounds__(kPersistentThreads)
    k_gather_persistent(const __grid_constant__ BatchPtrs ptrs, const JobDesc* __restrict__ jobs,
                        const TileDesc* __restrict__ tiles, int ntiles, unsigned* counter,
                        int stage_bytes, int nstages) {
  extern __shared__ __align__(128) unsigned char smem[];
  TileInfo* infos = reinterpret_cast<TileInfo*>(smem + (size_t)nstages * stage_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)nstages * (stage_bytes + kInfoBytes));
  uint64_t* empty = full + nstages;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), kConsumerWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ---- producer warp
    int it = 0;
    for (;; ++it) {
      const int s = it % nstages;
      const uint32_t fb = smem_addr(&full[s]);
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
      int t = 0;
      if (lane == 0) t = (int)atomicAdd(counter, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= ntiles) {
        if (lane == 0) {
          infos[s].tile = -1;
          mbar_arrive(fb);
        }
        ++it;
        break;
      }
      const TileDesc td = tiles[t];
      const JobDesc jd = jobs[td.job];
      const unsigned char* in_arr = ptrs.in[jd.arr];
      const unsigned char* in_depth = in_arr + jd.off_bytes;
      unsigned char* out_depth = ptrs.out[jd.arr] + jd.off_bytes;
      const unsigned char* safe_end = in_arr + (ptrs.in_bytes[jd.arr] & ~15ull);
      if (lane == 0) make_tile_info(infos[s], t, td, jd, in_depth, out_depth);
      __syncwarp();
      issue_tile_loads(td, jd, in_depth, safe_end, smem + (size_t)s * stage_bytes, fb, lane);
    }
    // make sure no copy into this CTA's shared memory is still in flight
    if (lane == 0) {
      const int armed = it;  // stages armed: iterations 0..it-1
      for (int s = 0; s < nstages && s < armed; ++s) {
        const int last = ((armed - 1 - s) / nstages) * nstages + s;  // last iteration using s
        const uint32_t par = (uint32_t)((last / nstages) & 1);
        mbar_wait_bounded(smem_addr(&full[s]), par, nullptr, kWaitLimitNs);
      }
    }
  } else {
    // ---- consumer warps
    const int ctid = tid - 32, nthr = 32 * kConsumerWarps;
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
      const TileInfo& ti = infos[s];
      if (ti.tile < 0) break;
      gather_store_dispatch(ti, smem + (size_t)s * stage_bytes, ctid, nthr);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
    }
  }
}

}  // namespace lfbp

// ====================================================================== host
using namespace lfbp;

struct lfbp_plan_s {
  int Nx = 0, Ny = 0, Nz = 0;
  std::vector<int> Ks, Kt;
  lfbp_dtype dt = LFBP_F32;
  lfbp_mode mode = LFBP_MAP_TRANSPOSE;
  int es = 4;
  std::vector<size_t> off;  // Nz + 1
  unsigned long long uid = 0;
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
};

Tuning default_tuning() {
  Tuning t;
  t.tile_bytes = env_int("LFBP_TILE_BYTES", 32768);
  t.ctas_per_sm = env_int("LFBP_CTAS_PER_SM", 2);
  t.stages = env_int("LFBP_STAGES", 0);
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

// One launch per depth of the plain kernel.
int run_plain(lfbp_plan p, const void* in, void* out, int mode, cudaStream_t st) {
  int rc = check_buffers(p, in, out);
  if (rc) return rc;
  const Tuning tu = default_tuning();
  const unsigned char* inb = (const unsigned char*)in;
  unsigned char* outb = (unsigned char*)out;
  const size_t arr_bytes = p->off.back() * (size_t)p->es;
  const unsigned char* safe_end = inb + (arr_bytes & ~(size_t)15);
  int max_smem = 0;
  for (int z = 0; z < p->Nz; ++z) {
    DepthTiling d = tile_depth(p->Ny, p->Ks[z], p->Kt[z], p->es, tu.tile_bytes);
    max_smem = std::max(max_smem, d.max_tile_bytes);
  }
  const int smem_total = max_smem + kInfoBytes + 16;
  if ((rc = ensure_smem_attr((const void*)k_gather_depth, smem_total))) return rc;
  for (int z = 0; z < p->Nz; ++z) {
    DepthTiling d = tile_depth(p->Ny, p->Ks[z], p->Kt[z], p->es, tu.tile_bytes);
    JobDesc jd;
    jd.off_bytes = p->off[z] * (size_t)p->es;
    jd.arr = 0;
    jd.Nx = p->Nx;
    jd.Ny = p->Ny;
    jd.Ks = p->Ks[z];
    jd.Kt = p->Kt[z];
    jd.es = p->es;
    jd.mode = mode;
    jd.pad = 0;
    dim3 grid(d.nV, p->Nx, d.nU);
    const int smem = d.max_tile_bytes;
    k_gather_depth<<<grid, kPlainThreads, smem + kInfoBytes + 16, st>>>(
        jd, inb + jd.off_bytes, safe_end, outb + jd.off_bytes, d.J, d.V, smem);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_gather_depth launch");
  return LFBP_OK;
}

// ---------------------------------------------------------------- batched --
struct BatchState {
  int dev = -1;
  std::vector<unsigned long long> uids;
  int ntiles = 0, njobs = 0;
  int stage_bytes = 0, nstages = 0, grid = 0, smem = 0;
  JobDesc* d_jobs = nullptr;
  TileDesc* d_tiles = nullptr;
  unsigned* d_counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  BatchPtrs ptrs;
  unsigned long long last_use = 0;
  ~BatchState() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_jobs) cudaFree(d_jobs);
    if (d_tiles) cudaFree(d_tiles);
    if (d_counter) cudaFree(d_counter);
  }
};

std::vector<std::unique_ptr<BatchState>> g_batches;  // guarded by g_mu
unsigned long long g_clock = 0;
constexpr size_t kMaxCachedBatches = 8;

int build_batch(BatchState& bs, int n, const lfbp_plan* plans, const Tuning& tu) {
  int sms = 0, optin = 0, dev = 0;
  int rc = device_props(&dev, &sms, &optin);
  if (rc) return rc;
  bs.dev = dev;
  std::vector<JobDesc> jobs;
  std::vector<TileDesc> tiles;
  int max_tile = 0;
  for (int i = 0; i < n; ++i) {
    lfbp_plan p = plans[i];
    for (int z = 0; z < p->Nz; ++z) {
      DepthTiling d = tile_depth(p->Ny, p->Ks[z], p->Kt[z], p->es, tu.tile_bytes);
      max_tile = std::max(max_tile, d.max_tile_bytes);
      JobDesc jd;
      jd.off_bytes = p->off[z] * (size_t)p->es;
      jd.arr = i;
      jd.Nx = p->Nx;
      jd.Ny = p->Ny;
      jd.Ks = p->Ks[z];
      jd.Kt = p->Kt[z];
      jd.es = p->es;
      jd.mode = (int)p->mode;
      jd.pad = 0;
      const unsigned job = (unsigned)jobs.size();
      jobs.push_back(jd);
      // u-block major, then p, then v-block: tiles in flight together touch
      // neighbouring input segments and neighbouring output runs
      for (int ub = 0; ub < d.nU; ++ub)
        for (int pp = 0; pp < p->Nx; ++pp)
          for (int vb = 0; vb < d.nV; ++vb) {
            TileDesc t;
            t.job = job;
            t.p = (unsigned short)pp;
            t.u0 = (unsigned short)(ub * d.J);
            t.v0 = (unsigned short)(vb * d.V);
            t.nrows = (unsigned short)std::min(d.J, p->Ks[z] - ub * d.J);
            t.ncols = (unsigned short)std::min(d.V, p->Kt[z] - vb * d.V);
            t.pad = 0;
            tiles.push_back(t);
          }
    }
  }
  bs.ntiles = (int)tiles.size();
  bs.njobs = (int)jobs.size();
  bs.stage_bytes = (max_tile + 127) & ~127;
  const int per_cta_budget = std::min(optin, (227 * 1024) / tu.ctas_per_sm - 1024);
  const int per_stage = bs.stage_bytes + kInfoBytes + 16;
  int nst = per_cta_budget / per_stage;
  if (tu.stages > 0) nst = std::min(nst, tu.stages);
  if (nst < 2) nst = std::min(2, optin / per_stage);
  if (nst < 1) return fail(LFBP_ERR_BAD_SHAPE, "tile does not fit in shared memory");
  bs.nstages = nst;
  bs.smem = nst * per_stage;
  bs.grid = sms * tu.ctas_per_sm;
  cudaError_t e;
  if (bs.njobs) {
    if ((e = cudaMalloc(&bs.d_jobs, sizeof(JobDesc) * jobs.size())) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(jobs)");
    if ((e = cudaMemcpy(bs.d_jobs, jobs.data(), sizeof(JobDesc) * jobs.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy(jobs)");
  }
  if (bs.ntiles) {
    if ((e = cudaMalloc(&bs.d_tiles, sizeof(TileDesc) * tiles.size())) != cudaSuccess)
      return cuda_fail(e, "cudaMalloc(tiles)");
    if ((e = cudaMemcpy(bs.d_tiles, tiles.data(), sizeof(TileDesc) * tiles.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy(tiles)");
  }
  if ((e = cudaMalloc(&bs.d_counter, 16)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(counter)");
  if ((rc = ensure_smem_attr((const void*)k_gather_persistent, bs.smem))) return rc;

  // graph: counter reset, then the persistent kernel
  if ((e = cudaGraphCreate(&bs.graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.dst = bs.d_counter;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 1;
  mp.height = 1;
  mp.pitch = 4;
  cudaGraphNode_t mnode;
  if ((e = cudaGraphAddMemsetNode(&mnode, bs.graph, nullptr, 0, &mp)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphAddMemsetNode");
  std::memset(&bs.ptrs, 0, sizeof(bs.ptrs));
  void* args[] = {&bs.ptrs, &bs.d_jobs, &bs.d_tiles, &bs.ntiles, &bs.d_counter, &bs.stage_bytes,
                  &bs.nstages};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = (void*)k_gather_persistent;
  kp.gridDim = dim3(bs.grid);
  kp.blockDim = dim3(kPersistentThreads);
  kp.sharedMemBytes = bs.smem;
  kp.kernelParams = args;
  if ((e = cudaGraphAddKernelNode(&bs.knode, bs.graph, &mnode, 1, &kp)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphAddKernelNode");
  if ((e = cudaGraphInstantiate(&bs.exec, bs.graph, 0)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphInstantiate");
  return LFBP_OK;
}

int run_batched(int n, const lfbp_plan* plans, const void* const* in, void* const* out,
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
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  BatchState* bs = nullptr;
  for (auto& b : g_batches) {
    if (b->dev != dev || (int)b->uids.size() != n) continue;
    bool same = true;
    for (int i = 0; i < n && same; ++i) same = b->uids[i] == plans[i]->uid;
    if (same) {
      bs = b.get();
      break;
    }
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
    int rc = build_batch(*nb, n, plans, default_tuning());
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
  if (std::memcmp(&np, &bs->ptrs, sizeof(np)) != 0) {
    bs->ptrs = np;
    void* args[] = {&bs->ptrs, &bs->d_jobs, &bs->d_tiles, &bs->ntiles, &bs->d_counter,
                    &bs->stage_bytes, &bs->nstages};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = (void*)k_gather_persistent;
    kp.gridDim = dim3(bs->grid);
    kp.blockDim = dim3(kPersistentThreads);
    kp.sharedMemBytes = bs->smem;
    kp.kernelParams = args;
    if ((e = cudaGraphExecKernelNodeSetParams(bs->exec, bs->knode, &kp)) != cudaSuccess)
      return cuda_fail(e, "cudaGraphExecKernelNodeSetParams");
  }
  if ((e = cudaGraphLaunch(bs->exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return LFBP_OK;
}

int make_plan(lfbp_plan* out, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
              lfbp_dtype dt, lfbp_mode mode) {
  if (!out) return fail(LFBP_ERR_NULL, "out is NULL");
  *out = nullptr;
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
    if (ks < 1 || kt < 1 || ks % 2 == 0 || kt % 2 == 0)
      return fail(LFBP_ERR_BAD_SHAPE, "every Ks and Kt must be odd and >= 1");
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

int lfbp_backproject_array(lfbp_plan p, const void* dH, void* dHp, void* cuda_stream) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  return run_plain(p, dH, dHp, (int)p->mode, (cudaStream_t)cuda_stream);
}

int lfbp_backproject_batched(int n, const lfbp_plan* plans, const void* const* dH,
                             void* const* dHp, void* cuda_stream) {
  return run_batched(n, plans, dH, dHp, (cudaStream_t)cuda_stream);
}

int lfbp_adjoint(lfbp_plan p, const void* dHp_grad, void* dH_grad, void* cuda_stream) {
  if (!p) return fail(LFBP_ERR_NULL, "plan is NULL");
  const int mode = p->mode == LFBP_MAP_TRANSPOSE ? 0 : 2;
  return run_plain(p, dHp_grad, dH_grad, mode, (cudaStream_t)cuda_stream);
}

int lfbp_sync_status(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int v = 0;
  if ((e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int))) != cudaSuccess)
    return cuda_fail(e, "read status");
  if (v != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
    return fail(v, "an in-kernel wait timed out; output incomplete");
  }
  return LFBP_OK;
}

const char* lfbp_last_error(void) { return t_err.c_str(); }

const char* lfbp_version(void) { return "lfbp 0.1 (sm_103a)"; }

}  // extern "C"
