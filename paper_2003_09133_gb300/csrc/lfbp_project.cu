// Projectors on a finite sensor / volume (fp32), used with H' by Richardson-Lucy
// style updates (Eq. 2) and by losses on backprojected volumes:
//
//   backprojection  g_z(X) = sum_{u,v} f(X-u+c_s, Y-v+c_t) * H'_z[(X-u+c_s) mod Nx][(Y-v+c_t) mod Ny][u][v]
//   forward (Eq. 1) f(S)   = sum_z sum_{s,t} g_z(S-s+c_s, .) * H_z[(S-s+c_s) mod Nx][..][s][t]
//
// Both are the same shift-variant sum  out(P) = sum_k in(P-k+c) * A[(P-k+c) mod N][k]
// (the cell of the *source* point selects the pattern), so one kernel serves both.
// Points outside the sensor / volume contribute nothing.  Lateral voxel grid =
// pixel grid; the cell position of a point P is P mod N.
//
// The backprojection also reads straight from H, without H' (substituting
// the map H'[p][q][u][v] = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]):
//   g_z(X) = sum_{s,t} f(X+s-c_s, Y+t-c_t) * H_z[X mod Nx][Y mod Ny][s][t],
// the sum  out(P) = sum_k in(P+k-c) * A[P mod N][k]  in which the cell of the
// *output* point selects the pattern (kOutCell below).
//
// Epilogues: store, accumulate (the forward sum over depths), and the
// Richardson-Lucy update of Eq. 2, out = g / norm * sum (0 where norm = 0).
//
// Gradient with respect to H' of a loss on g = H' f, given dL/dg:
//   dL/dH'_z[p][q][u][v] = sum over pixels S = (p + Nx i, q + Ny j) of f(S) * dL/dg_z(S + (u-c_s, v-c_t)).
//
// Every output element is produced by exactly one thread in a fixed order:
// results are deterministic (no atomics).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "lfbp_device.cuh"
#include "lfbp_project.h"

namespace lfbp {

constexpr int kSvTI = 8, kSvTJ = 32;  // outputs per block of the shift-variant sum
constexpr int kSvUC = 4;              // tap rows staged per step

__device__ __forceinline__ int pmod(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// Block: one output phase (rx, ry) = (X mod Nx, Y mod Ny) and a kSvTI x kSvTJ
// tile of outputs of that phase, X = rx + Nx*(i0+i), Y = ry + Ny*(j0+j).  For
// every tap (u, v) the pattern cell -- ((rx-u+c_s) mod Nx, (ry-v+c_t) mod Ny)
// for the source-cell sum, (rx, ry) for the output-cell sum -- is the same for
// the whole block, so the weights of kSvUC tap rows are staged in shared
// memory and broadcast.
template <bool kOutCell, int kEpi>
__global__ void __launch_bounds__(kSvTI* kSvTJ)
    k_shift_variant_sum(const float* __restrict__ A, int Nx, int Ny, int Ks, int Kt,
                        const float* __restrict__ in, int Wx, int Wy, float* out,
                        const float* g, const float* __restrict__ norm, int nI, int nJ) {
  extern __shared__ float ws[];  // [kSvUC][Kt]
  int b = blockIdx.x;
  const int tj = b % nJ;
  b /= nJ;
  const int ti = b % nI;
  b /= nI;
  const int ry = b % Ny;
  const int rx = b / Ny;
  const int i = threadIdx.y, j = threadIdx.x;
  const int tid = i * kSvTJ + j, nthr = kSvTI * kSvTJ;
  const int X = rx + Nx * (ti * kSvTI + i), Y = ry + Ny * (tj * kSvTJ + j);
  const bool active = X < Wx && Y < Wy;
  const int cs = (Ks - 1) / 2, ct = (Kt - 1) / 2;
  // taps whose input point lies inside the input:
  //   source-cell sum: 0 <= X-u+cs < Wx, 0 <= Y-v+ct < Wy
  //   output-cell sum: 0 <= X+u-cs < Wx, 0 <= Y+v-ct < Wy
  const int u_lo = kOutCell ? max(0, cs - X) : max(0, X + cs - Wx + 1);
  const int u_hi = kOutCell ? min(Ks - 1, Wx - 1 - X + cs) : min(Ks - 1, X + cs);
  const int v_lo = kOutCell ? max(0, ct - Y) : max(0, Y + ct - Wy + 1);
  const int v_hi = kOutCell ? min(Kt - 1, Wy - 1 - Y + ct) : min(Kt - 1, Y + ct);
  float acc = 0.f;
  for (int u0 = 0; u0 < Ks; u0 += kSvUC) {
    const int uc = min(kSvUC, Ks - u0);
    __syncthreads();
    for (int e = tid; e < uc * Kt; e += nthr) {
      const int du = e / Kt, v = e - du * Kt, u = u0 + du;
      const int p = kOutCell ? rx : pmod(rx - u + cs, Nx);
      const int q = kOutCell ? ry : pmod(ry - v + ct, Ny);
      ws[e] = __ldg(A + ((((size_t)p * Ny + q) * Ks + u) * Kt + v));
    }
    __syncthreads();
    if (!active) continue;
    const int ua = max(u0, u_lo), ub = min(u0 + uc - 1, u_hi);
    for (int u = ua; u <= ub; ++u) {
      const float* wrow = ws + (u - u0) * Kt;
      if (kOutCell) {
        const float* irow = in + (size_t)(X + u - cs) * Wy + (Y - ct);
        for (int v = v_lo; v <= v_hi; ++v) acc = fmaf(__ldg(irow + v), wrow[v], acc);
      } else {
        const float* irow = in + (size_t)(X - u + cs) * Wy + (Y + ct);
        for (int v = v_lo; v <= v_hi; ++v) acc = fmaf(__ldg(irow - v), wrow[v], acc);
      }
    }
  }
  if (active) {
    const size_t o = (size_t)X * Wy + Y;
    if (kEpi == kEpiStore) {
      out[o] = acc;
    } else if (kEpi == kEpiAccumulate) {
      out[o] += acc;
    } else {  // Eq. 2: g / (H'1) * [H' r]; each thread reads only its own g, so out may be g
      const float n = norm[o];
      out[o] = n != 0.f ? (g[o] / n) * acc : 0.f;
    }
  }
}

// ------------------------------------------------------------- phase conv --
// The output-cell sum  out(P) = sum_{u,v} in(P + (u,v) - c) * w_{P mod N}[u][v]
// serves every projection:
//   backprojection g = H' f:  w_{p,q} = H[p][q]                (read directly)
//   forward f = H g (Eq. 1):  w_{p,q} = H'[p][q]
//                            = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]
// (the map of Sec. 4 applied while the weights are staged; with H' at hand
// the roles swap, the map being its own inverse).  So neither projection
// needs the other array, and a block's weights are one pattern.
//
// Block: one output phase (px, py) and a (8*RI) x kPcTJ tile of its outputs
// X = px + Nx*i, Y = py + Ny*j.  The taps split by input phase: u = Nx*sigma + rho,
// v = Ny*upsilon + tau.  For each (rho, tau) the inputs form a dense subgrid
//   I(a, b) = in(Nx*(i0+a) + px + rho - c_s, Ny*(j0+b) + py + tau - c_t)
// and out(i, j) += sum_{sigma,upsilon} I(i-i0+sigma, j-j0+upsilon) * w[Nx sigma+rho][Ny upsilon+tau]:
// a dense correlation with an at most S x S kernel.  The subgrid tile and the
// sub-kernel (zero-padded to S x S) are staged in shared memory; each thread
// accumulates RI/2 rows x 4 columns of outputs in registers (half a warp per
// row group), reusing each loaded input row for every kernel row it meets.
// Terms are summed in a fixed order (deterministic); padded taps add exact
// zeros.  The subgrid arrives by TMA from the input laid out by phase, or by
// 4-byte cp.async copies (see the staging sections below).
constexpr int kPcThreads = 256;
constexpr int kPcTJ = 64;                // output columns per block (4 per lane, 16 lanes)
constexpr int kPcMaxDepths = 64;

struct PcDepth {
  long long off;  // element offset of the depth in A
  int Ks, Kt;
  int z;          // depth index: in + z*in_zstride, out/g/norm + z*out_zstride
  int pad;
};

struct PcArgs {
  CUtensorMap tmap;   // phase planes of `in` (TMA path): dims {Pjp, Pi, planes}
  CUtensorMap tmap2;  // phase planes of `g` (the gradient's dL/dg, TMA path)
  int* status;       // device status word (a wait that ran out: LFBP_ERR_TIMEOUT)
  int fault;         // 1 (LFBP_FAULT=stall, tests of the timeout path): TMA copies
                     // register their bytes on the barrier but are not issued
  int gsplit;        // k_phase_grad_pipe: blocks per (cell, depth), each a share of
                     // its (rho, tau) sub-problems (0 or 1: one block)
  const float* A;
  const float* in;
  long long in_zstride;
  float* out;
  long long out_zstride;
  const float* g;
  const float* norm;
  int Nx, Ny, Wx, Wy;
  int nTI, nTJ;
  int ndepth;
  int mapped;      // 1: weights through the map (see above)
  int sum_depths;  // 1: every block sums all depths of d[] into one output
  int epi;
  PcDepth d[kPcMaxDepths];
};

// 4-byte asynchronous copy global -> shared; with valid = false nothing is
// read and the destination is zero-filled (`src` must still be a valid address).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Sub-problem: depth di, input phase (rho, tau), with the quantities its
// staging needs kept up to date incrementally (no division per sub-problem):
// xoff = px + rho - c_s, yoff = py + tau - c_t, their cell positions
// ar = xoff mod Nx, br = yoff mod Ny, and the taps of the phase,
// Ssig = ceil((Ks - rho) / Nx) = Ks / Nx + [rho < Ks mod Nx] (rho < Nx), Sups likewise.
struct PcSub {
  int di, rho, tau;
  int Ks, Kt;
  int xoff, yoff, ar, br;
  int Ssig, Sups;
  int qs, ms, qt, mt;  // Ks / Nx, Ks mod Nx, Kt / Ny, Kt mod Ny
  int qx, qy;          // floor(xoff / Nx), floor(yoff / Ny): the subgrid's offset in its phase plane
};

__device__ __forceinline__ void pc_sub_depth(PcSub& c, int di, int Ks, int Kt, int px, int py,
                                             int Nx, int Ny) {
  c.di = di;
  c.rho = c.tau = 0;
  c.Ks = Ks;
  c.Kt = Kt;
  c.xoff = px - (Ks - 1) / 2;
  c.yoff = py - (Kt - 1) / 2;
  c.ar = pmod(c.xoff, Nx);
  c.br = pmod(c.yoff, Ny);
  c.qx = (c.xoff - c.ar) / Nx;
  c.qy = (c.yoff - c.br) / Ny;
  c.qs = Ks / Nx;
  c.ms = Ks - c.qs * Nx;
  c.qt = Kt / Ny;
  c.mt = Kt - c.qt * Ny;
  c.Ssig = c.qs + (c.ms > 0);
  c.Sups = c.qt + (c.mt > 0);
}

// Next (rho, tau) of the same depth; false after the last one.
__device__ __forceinline__ bool pc_sub_next_phase(PcSub& c, int px, int py, int Nx, int Ny) {
  if (c.tau + 1 < Ny && c.tau + 1 < c.Kt) {
    ++c.tau;
    ++c.yoff;
    if (++c.br == Ny) {
      c.br = 0;
      ++c.qy;
    }
    c.Sups = c.qt + (c.tau < c.mt);
    return true;
  }
  if (c.rho + 1 < Nx && c.rho + 1 < c.Ks) {
    ++c.rho;
    ++c.xoff;
    if (++c.ar == Nx) {
      c.ar = 0;
      ++c.qx;
    }
    c.Ssig = c.qs + (c.rho < c.ms);
    c.tau = 0;
    c.yoff = py - (c.Kt - 1) / 2;
    c.br = pmod(c.yoff, Ny);
    c.qy = (c.yoff - c.br) / Ny;
    c.Sups = c.qt + (c.mt > 0);
    return true;
  }
  return false;
}

// Copies of the input subgrid I(r, col) = in(Nx*(i0+r) + xoff, Ny*(j0+col) + yoff),
// r < IR, col < ICP (zero outside the sensor / volume and for col >= IC) into
// dst[r * ICP + col]; warp wi takes rows wi, wi+8, ..., lane the columns
// lane + 32 k.  Row and column tests and offsets are formed once per row and
// once per column.
template <int IR, int IC, int ICP, int UR = (IR + 7) / 8>
__device__ __forceinline__ void pc_stage_input(float* dst, const float* inz, const float* dummy,
                                               int Nx, int Ny, int Wx, int Wy, int i0, int j0,
                                               int xoff, int yoff, int wi, int lane) {
  constexpr int KC = (ICP + 31) / 32;
  int yk[KC];
  bool okc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    yk[k] = Ny * (j0 + lane + 32 * k) + yoff;
    okc[k] = lane + 32 * k < IC && yk[k] >= 0 && yk[k] < Wy;
  }
  int x = Nx * (i0 + wi) + xoff;
#pragma unroll UR
  for (int rr = 0; rr < (IR + 7) / 8; ++rr) {
    const int r = wi + 8 * rr;
    if (r < IR) {
      const bool xin = x >= 0 && x < Wx;
      const float* row = inz + (long long)(xin ? x : 0) * Wy;
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        if (k + 1 < KC || lane + 32 * k < ICP) {
          const bool ok = xin && okc[k];
          cp_async4(dst + r * ICP + lane + 32 * k, ok ? row + yk[k] : dummy, ok);
        }
      }
    }
    x += 8 * Nx;
  }
}

// ------------------------------------------------------------ TMA staging --
// On the TMA path a projection's input is first laid out by phase (planes,
// k_phase_planes below): plane (z, rx, ry) holds in_z(Nx*i + rx, Ny*j + ry)
// at [i][j], zero outside the sensor / volume.  A sub-problem's subgrid
// I(r, col) = in(Nx*(i0+r) + xoff, Ny*(j0+col) + yoff) is then the box of
// plane (z, xoff mod Nx, yoff mod Ny) at rows i0 + floor(xoff/Nx) + r and
// columns j0 + floor(yoff/Ny) + col, moved by one TMA tensor copy; rows and
// columns outside the plane arrive as zeros.  The box starts at the
// 16-byte-aligned column below, REM = floor(yoff/Ny) mod 4 columns early, and
// the compute reads from column REM on.
constexpr uint64_t kPcWaitNs = 2000000000ull;  // 2 s per in-kernel wait

template <int S>
struct PcBox {
  // a lane's 16-byte reads start at b0 <= 60 and cover REM + S + 3 <= S + 6 columns
  static constexpr int BX = (kPcTJ + S + 5 + 3) & ~3;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Thread 0: the TMA copy of sub-problem c's subgrid (plane z0 + (ar, br)) into
// `dst`, completing on `bar` (one arrival plus the box's bytes).
__device__ __forceinline__ void pc_tma_stage(const PcArgs& a, const PcSub& c, int zplane0,
                                             float* dst, uint64_t* bar, int i0, int j0,
                                             uint32_t bytes) {
  fence_proxy_async_smem();  // the buffer's previous (generic) reads come first
  const uint32_t b = smem_addr(bar);
  mbar_expect_tx(b, bytes);
  if (!a.fault)
    tma_load_3d(smem_addr(dst), &a.tmap, j0 + c.qy - (c.qy & 3), i0 + c.qx,
                (zplane0 + c.ar) * a.Ny + c.br, b);
  mbar_arrive(b);
}

// The same copy for a barrier whose arrivals come from elsewhere (only the
// expected bytes are registered here).
__device__ __forceinline__ void pc_tma_stage_noarrive(const PcArgs& a, const PcSub& c, int zplane0,
                                                      float* dst, uint64_t* bar, int i0, int j0,
                                                      uint32_t bytes) {
  fence_proxy_async_smem();
  const uint32_t b = smem_addr(bar);
  mbar_expect_tx(b, bytes);
  if (!a.fault)
    tma_load_3d(smem_addr(dst), &a.tmap, j0 + c.qy - (c.qy & 3), i0 + c.qx,
                (zplane0 + c.ar) * a.Ny + c.br, b);
}

// Products of one staged sub-problem: rows r of the subgrid tile (pitch PITCH,
// data from column REM on) against the S x S sub-kernel, into acc.
template <int S, int RH, int REM, int PITCH, int NACC>
__device__ __forceinline__ void pc_products(const float* Ib, const float* const* wbs, int a0, int b0,
                                            float (&acc)[NACC][RH][4]) {
  constexpr int S4 = (S + 3) & ~3;
  constexpr int NC4 = (REM + S + 3 + 3) / 4;
#pragma unroll
  for (int r = 0; r < RH + S - 1; ++r) {
    float xv[4 * NC4];
    const float* src = Ib + (a0 + r) * PITCH + b0;
#pragma unroll
    for (int c4 = 0; c4 < NC4; ++c4) {
      const float4 p = *reinterpret_cast<const float4*>(src + 4 * c4);
      xv[4 * c4] = p.x;
      xv[4 * c4 + 1] = p.y;
      xv[4 * c4 + 2] = p.z;
      xv[4 * c4 + 3] = p.w;
    }
#pragma unroll
    for (int d = 0; d < NACC; ++d) {
      const float* wb = wbs[d];
#pragma unroll
      for (int sg = 0; sg < S; ++sg) {
        const int ai = r - sg;
        if (ai < 0 || ai >= RH) continue;
        float wr[S4];  // the kernel row sg, in 16-byte shared loads
#pragma unroll
        for (int u4 = 0; u4 < S4 / 4; ++u4) {
          const float4 w4 = *reinterpret_cast<const float4*>(wb + sg * S4 + 4 * u4);
          wr[4 * u4] = w4.x;
          wr[4 * u4 + 1] = w4.y;
          wr[4 * u4 + 2] = w4.z;
          wr[4 * u4 + 3] = w4.w;
        }
#pragma unroll
        for (int up = 0; up < S; ++up) {
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[d][ai][c] = fmaf(xv[REM + up + c], wr[up], acc[d][ai][c]);
        }
      }
    }
  }
}

template <int S, int RH, int PITCH, int NACC>
__device__ __forceinline__ void pc_products_rem(int rem, const float* Ib, const float* const* wbs,
                                                int a0, int b0, float (&acc)[NACC][RH][4]) {
  switch (rem) {
    case 0: pc_products<S, RH, 0, PITCH, NACC>(Ib, wbs, a0, b0, acc); break;
    case 1: pc_products<S, RH, 1, PITCH, NACC>(Ib, wbs, a0, b0, acc); break;
    case 2: pc_products<S, RH, 2, PITCH, NACC>(Ib, wbs, a0, b0, acc); break;
    default: pc_products<S, RH, 3, PITCH, NACC>(Ib, wbs, a0, b0, acc); break;
  }
}

// A wait that ran out: record it, let this thread's copies land, and tell the
// caller to return (every thread of the block takes the same branch).
__device__ __forceinline__ bool pc_abort(const PcArgs& a, bool timed_out) {
  if (!__syncthreads_or(timed_out)) return false;
  if (threadIdx.x == 0 && a.status) atomicCAS(a.status, 0, kStatusTimeout);
  cp_async_wait<0>();
  return true;
}

// cp.async copies of this thread so far arrive on `bar` when they land (the
// arrival counts toward the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

constexpr int kPcStages = 3;                    // input/weight stages of the pipelined kernel
constexpr int kPcPipeThreads = kPcThreads + 32;  // 8 consumer warps + 1 producer warp

// The TMA path of k_phase_conv as a producer/consumer pipeline without
// block-wide barriers.  Warp 8 produces: per sub-problem it issues the weights
// as 4-byte cp.async copies, lane by lane, and each lane's copies arrive on the
// stage's full barrier when they land.  Lane 0 also issues the TMA copy of the
// input subgrid and writes the stage's column remainder, releasing it with a
// plain arrival.  Warps 0-7 consume the stages in order and release each one
// with a per-warp arrival on its empty barrier.  Same products in the same
// order as k_phase_conv.
// DB = 1: one depth per block (grid.y), or all depths summed (sum_depths);
// DB > 1: DB depths of one cut-out size reading one shared image, each staged
// subgrid feeding all DB depths' weights (the backprojections).
template <int S, int RI, int DB, int NST = kPcStages>
__global__ void __launch_bounds__(kPcPipeThreads) k_phase_conv_pipe(const __grid_constant__ PcArgs a) {
  constexpr int TI = 8 * RI;
  constexpr int S4 = (S + 3) & ~3;
  constexpr int IR = TI + S - 1;
  constexpr int RH = RI / 2;
  constexpr int ICP = PcBox<S>::BX;
  constexpr int IB = (IR * ICP + 31) & ~31;
  constexpr int NW = DB * S * S4;  // weights per stage
  __shared__ __align__(128) float I_s[NST][IB];
  __shared__ __align__(16) float w_s[NST][NW];
  __shared__ int rem_s[NST];
  __shared__ __align__(8) uint64_t full[NST], empty[NST];
  __shared__ int abort_flag;
  const int Nx = a.Nx, Ny = a.Ny, Wx = a.Wx, Wy = a.Wy;
  int t = blockIdx.x;
  const int tj = t % a.nTJ;
  t /= a.nTJ;
  const int ti = t % a.nTI;
  t /= a.nTI;
  const int py = t % Ny, px = t / Ny;
  const int i0 = ti * TI, j0 = tj * kPcTJ;
  const int tid = threadIdx.x, wi = tid >> 5, lane = tid & 31;
  // DB = 1: depths d_lo .. d_hi-1 in sequence; DB > 1: the group dbase .. dbase+nd-1 at once
  const int dbase = DB > 1 ? (int)blockIdx.y * DB : 0;
  const int nd = DB > 1 ? min(DB, a.ndepth - dbase) : 1;
  const int d_lo = DB > 1 ? dbase : a.sum_depths ? 0 : (int)blockIdx.y;
  const int d_hi = DB > 1 ? dbase + 1 : a.sum_depths ? a.ndepth : (int)blockIdx.y + 1;
  int nsub = 0;
  for (int d = d_lo; d < d_hi; ++d) nsub += min(Nx, a.d[d].Ks) * min(Ny, a.d[d].Kt);
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_addr(&full[s]), 33);  // 32 copy-completion arrivals + lane 0's release
      mbar_init(smem_addr(&empty[s]), 8);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (wi == 8) {
    // ---- producer warp
    PcSub c;
    pc_sub_depth(c, d_lo, a.d[d_lo].Ks, a.d[d_lo].Kt, px, py, Nx, Ny);
    int issued = 0;
    for (int k = 0; k < nsub; ++k) {
      const int s = k % NST;
      if (k >= NST &&
          !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)((k / NST - 1) & 1), &abort_flag,
                             kPcWaitNs)) {
        if (lane == 0) {
          abort_flag = 1;
          if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
        }
        break;
      }
      const int Ks = c.Ks, Kt = c.Kt;
      for (int e = lane; e < NW; e += 32) {
        const int wd = e / (S * S4), ee = e - wd * (S * S4);
        const int sg = ee / S4, up = ee - sg * S4;
        const bool ok = wd < nd && sg < c.Ssig && up < c.Sups;
        const int u = Nx * sg + c.rho, v = Ny * up + c.tau;
        const float* Az = a.A + (ok ? a.d[DB > 1 ? dbase + wd : c.di].off : 0);
        const float* src =
            !ok ? a.A
                : a.mapped ? Az + (((size_t)c.ar * Ny + c.br) * Ks + (Ks - 1 - u)) * Kt + (Kt - 1 - v)
                           : Az + (((size_t)px * Ny + py) * Ks + u) * Kt + v;
        cp_async4(&w_s[s][e], src, ok);
      }
      if (lane == 0) {
        rem_s[s] = c.qy & 3;
        const int zp = (DB == 1 && a.in_zstride) ? a.d[c.di].z * Nx : 0;
        pc_tma_stage_noarrive(a, c, zp, I_s[s], &full[s], i0, j0,
                              (uint32_t)(IR * ICP * sizeof(float)));
      }
      cp_async_arrive_noinc(&full[s]);  // this lane's arrival, once its copies have landed
      if (lane == 0) mbar_arrive(smem_addr(&full[s]));  // releases rem_s[s]
      ++issued;
      if (k + 1 < nsub && !pc_sub_next_phase(c, px, py, Nx, Ny))
        pc_sub_depth(c, c.di + 1, a.d[c.di + 1].Ks, a.d[c.di + 1].Kt, px, py, Nx, Ny);
    }
    // nothing of this CTA may still be landing when it exits: wait for the
    // stages still in flight (already complete unless the consumers gave up;
    // none were issued under the stall injection)
    if (lane == 0 && !a.fault)
      for (int j = issued - 1; j >= 0 && j >= issued - NST; --j)
        mbar_wait_bounded(smem_addr(&full[j % NST]), (uint32_t)((j / NST) & 1), nullptr,
                          kPcWaitNs);
    cp_async_wait<0>();
    return;
  }

  // ---- consumer warps
  const int a0 = wi * RI + (lane >> 4) * RH, b0 = 4 * (lane & 15);
  float acc[DB][RH][4];
#pragma unroll
  for (int d = 0; d < DB; ++d)
#pragma unroll
    for (int i = 0; i < RH; ++i) acc[d][i][0] = acc[d][i][1] = acc[d][i][2] = acc[d][i][3] = 0.f;
  for (int k = 0; k < nsub; ++k) {
    const int s = k % NST;
    if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)((k / NST) & 1), &abort_flag,
                           kPcWaitNs)) {
      if (lane == 0) {
        abort_flag = 1;
        if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
      }
      return;
    }
    const float* wbs[DB];
#pragma unroll
    for (int d = 0; d < DB; ++d) wbs[d] = w_s[s] + d * (S * S4);
    pc_products_rem<S, RH, ICP, DB>(rem_s[s], I_s[s], wbs, a0, b0, acc);
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
  }

#pragma unroll
  for (int d = 0; d < DB; ++d) {
    if (d >= nd) break;
    const long long zo = DB > 1 ? (long long)a.d[dbase + d].z * a.out_zstride
                         : a.sum_depths ? 0 : (long long)a.d[blockIdx.y].z * a.out_zstride;
#pragma unroll
    for (int i = 0; i < RH; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int X = px + Nx * (i0 + a0 + i), Y = py + Ny * (j0 + b0 + c);
        if (X >= Wx || Y >= Wy) continue;
        const long long o = zo + (long long)X * Wy + Y;
        if (a.epi == kEpiStore) {
          a.out[o] = acc[d][i][c];
        } else if (a.epi == kEpiAccumulate) {
          a.out[o] += acc[d][i][c];
        } else {
          const float n = a.norm[o];
          a.out[o] = n != 0.f ? (a.g[o] / n) * acc[d][i][c] : 0.f;
        }
      }
  }
}

// RI: output rows per thread; the block (8 warps) covers 8*RI rows x 64 columns.
// The sub-problems (depth, rho, tau) run through a two-buffer pipeline: the
// copies of the next one are in flight while the current one is computed.
// kTma: the input subgrid arrives by one TMA tensor copy from the phase planes
// (a.tmap); otherwise by the 4-byte cp.async staging above.
template <int S, int RI, bool kTma>
__global__ void __launch_bounds__(kPcThreads) k_phase_conv(const __grid_constant__ PcArgs a) {
  constexpr int TI = 8 * RI;
  constexpr int S4 = (S + 3) & ~3;   // weight row pitch
  constexpr int IR = TI + S - 1;     // subgrid rows
  constexpr int RH = RI / 2;         // output rows per thread (half a warp per row group)
  constexpr int IC = kPcTJ + S + 3;  // subgrid columns (lane cols 4l .. 4l+S+2, read in fours)
  constexpr int ICP = kTma ? PcBox<S>::BX : (IC + 3) & ~3;  // 16-byte aligned rows
  constexpr int IB = (IR * ICP + 31) & ~31;  // buffer stride: 128-byte aligned TMA destinations
  __shared__ __align__(16) float w_s[2][S * S4];
  __shared__ __align__(128) float I_s[2][IB];
  __shared__ __align__(8) uint64_t full[2];
  const int Nx = a.Nx, Ny = a.Ny, Wx = a.Wx, Wy = a.Wy;
  int t = blockIdx.x;
  const int tj = t % a.nTJ;
  t /= a.nTJ;
  const int ti = t % a.nTI;
  t /= a.nTI;
  const int py = t % Ny, px = t / Ny;
  const int i0 = ti * TI, j0 = tj * kPcTJ;
  const int tid = threadIdx.x, wi = tid >> 5, lane = tid & 31;
  // lanes 0-15 and 16-31 take the two halves of the warp's RI rows; 4 columns each
  const int a0 = wi * RI + (lane >> 4) * RH, b0 = 4 * (lane & 15);
  const int d_lo = a.sum_depths ? 0 : (int)blockIdx.y;
  const int d_hi = a.sum_depths ? a.ndepth : (int)blockIdx.y + 1;
  if (kTma) {
    if (tid == 0) {
      mbar_init(smem_addr(&full[0]), 1);
      mbar_init(smem_addr(&full[1]), 1);
      fence_mbar_init();
    }
    __syncthreads();
  }

  static_assert(S * S4 <= kPcThreads, "one weight per thread");
  // issue the copies of sub-problem c into buffer buf (one commit group)
  auto stage = [&](const PcSub& c, int buf) {
    const PcDepth& dd = a.d[c.di];
    const int Ks = c.Ks, Kt = c.Kt;
    if (tid < S * S4) {
      const int sg = tid / S4, up = tid - sg * S4;
      const bool ok = sg < c.Ssig && up < c.Sups;
      const int u = Nx * sg + c.rho, v = Ny * up + c.tau;
      const float* Az = a.A + dd.off;
      const float* src =
          !ok ? a.A
              : a.mapped ? Az + (((size_t)c.ar * Ny + c.br) * Ks + (Ks - 1 - u)) * Kt + (Kt - 1 - v)
                         : Az + (((size_t)px * Ny + py) * Ks + u) * Kt + v;
      cp_async4(&w_s[buf][tid], src, ok);
    }
    if (kTma) {
      if (tid == 0)
        pc_tma_stage(a, c, (a.in_zstride ? dd.z : 0) * Nx, I_s[buf], &full[buf], i0, j0,
                     (uint32_t)(IR * ICP * sizeof(float)));
    } else {
      pc_stage_input<IR, IC, ICP>(I_s[buf], a.in + (long long)dd.z * a.in_zstride, a.in, Nx, Ny,
                                  Wx, Wy, i0, j0, c.xoff, c.yoff, wi, lane);
    }
    cp_async_commit();
  };
  auto advance = [&](PcSub& c) -> bool {  // next sub-problem; false at the end
    if (pc_sub_next_phase(c, px, py, Nx, Ny)) return true;
    if (c.di + 1 >= d_hi) return false;
    pc_sub_depth(c, c.di + 1, a.d[c.di + 1].Ks, a.d[c.di + 1].Kt, px, py, Nx, Ny);
    return true;
  };

  float acc[1][RH][4];
#pragma unroll
  for (int i = 0; i < RH; ++i) acc[0][i][0] = acc[0][i][1] = acc[0][i][2] = acc[0][i][3] = 0.f;
  PcSub cur;
  pc_sub_depth(cur, d_lo, a.d[d_lo].Ks, a.d[d_lo].Kt, px, py, Nx, Ny);
  PcSub nxt = cur;
  bool more = advance(nxt);
  stage(cur, 0);
  for (int k = 0;; ++k) {
    const int buf = k & 1;
    if (more)
      stage(nxt, buf ^ 1);
    else
      cp_async_commit();  // keep the group count uniform
    cp_async_wait<1>();   // the current buffer's weights have landed (this thread's copies);
                          // the block barrier in pc_abort (TMA) or below publishes them
    if (kTma) {
      const bool ok = mbar_wait_bounded(smem_addr(&full[buf]), (uint32_t)((k >> 1) & 1), nullptr,
                                        kPcWaitNs);
      if (pc_abort(a, !ok)) {
        if (tid == 0 && more)  // the copy into the other buffer
          mbar_wait_bounded(smem_addr(&full[buf ^ 1]), (uint32_t)(((k + 1) >> 1) & 1), nullptr,
                            kPcWaitNs);
        return;
      }
    } else {
      __syncthreads();  // ... and everybody's
    }
    const float* wbs[1] = {w_s[buf]};
    if (kTma)
      pc_products_rem<S, RH, ICP, 1>(cur.qy & 3, I_s[buf], wbs, a0, b0, acc);
    else
      pc_products<S, RH, 0, ICP, 1>(I_s[buf], wbs, a0, b0, acc);
    __syncthreads();  // buffer buf is free for the copies issued next round
    if (!more) break;
    cur = nxt;
    more = advance(nxt);
  }
  cp_async_wait<0>();

  const long long zo = a.sum_depths ? 0 : (long long)a.d[blockIdx.y].z * a.out_zstride;
#pragma unroll
  for (int i = 0; i < RH; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int X = px + Nx * (i0 + a0 + i), Y = py + Ny * (j0 + b0 + c);
      if (X >= Wx || Y >= Wy) continue;
      const long long o = zo + (long long)X * Wy + Y;
      if (a.epi == kEpiStore) {
        a.out[o] = acc[0][i][c];
      } else if (a.epi == kEpiAccumulate) {
        a.out[o] += acc[0][i][c];
      } else {
        const float n = a.norm[o];
        a.out[o] = n != 0.f ? (a.g[o] / n) * acc[0][i][c] : 0.f;
      }
    }
}

// ------------------------------------------------------------- phase grad --
// dL/dH'_z[p][q][u][v] = sum over pixels S = (p + Nx i, q + Ny j) of f(S) * dg_z(S + (u,v) - c).
// Split the taps by phase, u = Nx*sigma + rho, v = Ny*upsilon + tau: with
//   F(i, j) = f(p + Nx i, q + Ny j),  G(a, b) = dg_z(Nx a + p + rho - c_s, Ny b + q + tau - c_t),
// the S x S outputs of one (rho, tau) are  O[sigma][upsilon] = sum_{i,j} F(i,j) G(i+sigma, j+upsilon).
// Block: one cell (p, q) of one depth; the cell's pixels in tiles of
// kGrI x kGrJ.  Per tile F is staged once; the G tiles of the (rho, tau)
// sub-problems run through a two-buffer cp.async pipeline.  Thread (i, sigma)
// walks row i of F and row i + sigma of G in steps of four columns (16-byte
// shared loads; a sliding window of G columns in registers) and sums its
// row's products for all upsilon; then the rows are reduced: a shuffle tree
// over a warp's 32 rows, then the two warps of each sigma in order
// (deterministic).  Tiles after the first add to the output.
constexpr int kGrI = 64, kGrJ = 64;

template <int S, bool kTma>
struct GradGeom {
  static constexpr int FP = kGrJ + 4;                      // F row pitch (= 4 mod 8: no conflicts)
  static constexpr int GR = kGrI + S - 1;                  // G tile rows
  // cp.async path: columns 0 .. GJ-1 from column 0; TMA path: the box starts up
  // to 3 columns early (REM) and a window of NWT columns covers REM + S + 3
  static constexpr int NW = 4 * ((S + 3 + 3) / 4);         // G window (columns) per step, REM = 0
  static constexpr int NWT = 4 * ((S + 6 + 3) / 4);        // ... for any REM < 4
  static constexpr int GJ0 = kTma ? kGrJ - 4 + NWT : (kGrJ + S - 1 + 3) & ~3;
  static constexpr int GP = (GJ0 % 8 == 4) ? GJ0 : GJ0 + 4;  // G row pitch (= 4 mod 8)
  static constexpr int GB = (GR * GP + 31) & ~31;          // G buffer stride (128-byte aligned)
  // + 128: the start is rounded up to a 128-byte boundary (TMA destinations)
  static constexpr size_t smem = sizeof(float) * (kGrI * FP + 2 * GB) + 128;
};

// Thread (row i, sigma)'s sums over one G tile: acc[up] = sum_j F(i, j) G(i + sigma, j + up),
// F row Fr, G row Gr (data from column REM on), 16-byte loads with a sliding
// window of NW G columns in registers.
template <int S, int REM, int NW>
__device__ __forceinline__ void grad_row(const float* Fr, const float* Gr, float (&acc)[S]) {
  float w[NW];
#pragma unroll
  for (int c4 = 0; c4 < NW / 4; ++c4) {
    const float4 g4 = *reinterpret_cast<const float4*>(Gr + 4 * c4);
    w[4 * c4] = g4.x;
    w[4 * c4 + 1] = g4.y;
    w[4 * c4 + 2] = g4.z;
    w[4 * c4 + 3] = g4.w;
  }
#pragma unroll
  for (int j4 = 0; j4 < kGrJ / 4; ++j4) {
    const float4 f4 = *reinterpret_cast<const float4*>(Fr + 4 * j4);
    const float fv[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int up = 0; up < S; ++up) acc[up] = fmaf(fv[c], w[REM + c + up], acc[up]);
    if (j4 + 1 < kGrJ / 4) {  // slide the window by four columns
#pragma unroll
      for (int t = 0; t < NW - 4; ++t) w[t] = w[t + 4];
      const float4 g4 = *reinterpret_cast<const float4*>(Gr + 4 * j4 + NW);
      w[NW - 4] = g4.x;
      w[NW - 3] = g4.y;
      w[NW - 2] = g4.z;
      w[NW - 1] = g4.w;
    }
  }
}

// kTma: F and the G tiles arrive by TMA tensor copies from the phase planes of
// f (a.tmap) and of dg (a.tmap2); otherwise by 4-byte cp.async copies.
template <int S, bool kTma>
__global__ void __launch_bounds__(256) k_phase_grad(const __grid_constant__ PcArgs a) {
  using Gm = GradGeom<S, kTma>;
  constexpr int FP = Gm::FP, GR = Gm::GR, GJ0 = Gm::GJ0, GP = Gm::GP, GB = Gm::GB;
  static_assert(kTma || kGrJ - 4 + Gm::NW <= GJ0, "window stays inside the staged columns");
  extern __shared__ __align__(128) float gsm_raw[];
  float* gsm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(gsm_raw) + 127) & ~uintptr_t(127));
  float* F_s = gsm;
  float* G_s = gsm + kGrI * FP;  // [2][GB]
  __shared__ float part[8][S];
  __shared__ __align__(8) uint64_t bars[3];  // G buffers 0, 1; F
  const int Nx = a.Nx, Ny = a.Ny, Wx = a.Wx, Wy = a.Wy;
  const int p = blockIdx.x / Ny, q = blockIdx.x % Ny;
  const PcDepth dd = a.d[blockIdx.y];
  const int Ks = dd.Ks, Kt = dd.Kt;
  const float* f = a.in;
  const float* dg = a.g + (long long)dd.z * a.out_zstride;
  float* dA = a.out + dd.off + ((long long)p * Ny + q) * Ks * Kt;
  const int nI = (Wx - p + Nx - 1) / Nx, nJ = (Wy - q + Ny - 1) / Ny;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i = tid & 63, sgs = tid >> 6;
  if (kTma) {
    if (tid == 0) {
      for (int b = 0; b < 3; ++b) mbar_init(smem_addr(&bars[b]), 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  // the G tile of sub-problem c into buffer buf
  auto stage_g = [&](const PcSub& c, int buf, int i0, int j0) {
    float* dst = G_s + buf * GB;
    if (kTma) {
      if (tid == 0) {
        fence_proxy_async_smem();
        const uint32_t b = smem_addr(&bars[buf]);
        mbar_expect_tx(b, (uint32_t)(GR * GP * sizeof(float)));
        if (!a.fault)
          tma_load_3d(smem_addr(dst), &a.tmap2, j0 + c.qy - (c.qy & 3), i0 + c.qx,
                      (dd.z * Nx + c.ar) * Ny + c.br, b);
        mbar_arrive(b);
      }
    } else {
      pc_stage_input<GR, GJ0, GP, 1>(dst, dg, dg, Nx, Ny, Wx, Wy, i0, j0, c.xoff, c.yoff, warp,
                                     lane);
    }
  };
  bool first_tile = true;
  int ng = 0;  // G tiles staged so far (buffer uses: parity of each buffer's barrier)
  int nf = 0;  // F tiles staged so far
  for (int i0 = 0; i0 < nI; i0 += kGrI)
    for (int j0 = 0; j0 < nJ; j0 += kGrJ) {
      __syncthreads();  // the previous tile's buffers are consumed
      if (kTma) {
        if (tid == 0) {
          fence_proxy_async_smem();
          const uint32_t b = smem_addr(&bars[2]);
          mbar_expect_tx(b, (uint32_t)(kGrI * FP * sizeof(float)));
          if (!a.fault) tma_load_3d(smem_addr(F_s), &a.tmap, j0, i0, p * Ny + q, b);
          mbar_arrive(b);
        }
      } else {
        pc_stage_input<kGrI, kGrJ, FP, 1>(F_s, f, f, Nx, Ny, Wx, Wy, i0, j0, p, q, warp, lane);
      }
      PcSub cur;
      pc_sub_depth(cur, 0, Ks, Kt, p, q, Nx, Ny);
      const int g0 = ng;  // this tile's first G tile goes to buffer g0 & 1
      stage_g(cur, g0 & 1, i0, j0);
      ++ng;
      cp_async_commit();
      for (int k = 0;; ++k) {
        const int buf = (g0 + k) & 1;
        PcSub nxt = cur;
        const bool more = pc_sub_next_phase(nxt, p, q, Nx, Ny);
        if (more) {
          stage_g(nxt, buf ^ 1, i0, j0);
          ++ng;
        }
        cp_async_commit();
        cp_async_wait<1>();
        if (kTma) {
          const bool okg = mbar_wait_bounded(smem_addr(&bars[buf]),
                                             (uint32_t)(((g0 + k) >> 1) & 1), nullptr, kPcWaitNs);
          const bool okf = k > 0 || mbar_wait_bounded(smem_addr(&bars[2]), (uint32_t)(nf & 1),
                                                      nullptr, kPcWaitNs);
          const bool ok = okg && okf;
          if (pc_abort(a, !ok)) {
            if (tid == 0 && more)
              mbar_wait_bounded(smem_addr(&bars[buf ^ 1]), (uint32_t)(((g0 + k + 1) >> 1) & 1),
                                nullptr, kPcWaitNs);
            return;
          }
        } else {
          __syncthreads();  // F and this sub-problem's G have landed
        }
        const float* Gb = G_s + buf * GB;
        const int rem = kTma ? (cur.qy & 3) : 0;
        for (int s0 = 0; s0 < S; s0 += 4) {
          const int sg = s0 + sgs;
          float acc[S];
#pragma unroll
          for (int up = 0; up < S; ++up) acc[up] = 0.f;
          if (sg < S) {
            const float* Fr = F_s + i * FP;
            const float* Gr = Gb + (i + sg) * GP;
            if (!kTma) {
              grad_row<S, 0, Gm::NW>(Fr, Gr, acc);
            } else {
              switch (rem) {
                case 0: grad_row<S, 0, Gm::NWT>(Fr, Gr, acc); break;
                case 1: grad_row<S, 1, Gm::NWT>(Fr, Gr, acc); break;
                case 2: grad_row<S, 2, Gm::NWT>(Fr, Gr, acc); break;
                default: grad_row<S, 3, Gm::NWT>(Fr, Gr, acc); break;
              }
            }
          }
          // rows of the warp: shuffle tree; then the two warps of each sigma
#pragma unroll
          for (int up = 0; up < S; ++up) {
            float v = acc[up];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[warp][up] = v;
          }
          __syncthreads();
          if (tid < 4 * S) {  // (sigma slot, upsilon): warps 2w and 2w+1 hold sigma s0 + w
            const int w2 = tid / S, up = tid - w2 * S, sgo = s0 + w2;
            if (sgo < cur.Ssig && up < cur.Sups) {
              const float v = part[2 * w2][up] + part[2 * w2 + 1][up];
              float* o = dA + (size_t)(Nx * sgo + cur.rho) * Kt + (Ny * up + cur.tau);
              *o = first_tile ? v : *o + v;
            }
          }
          __syncthreads();  // part and (after the last round) buffer buf are free
        }
        if (!more) break;
        cur = nxt;
      }
      cp_async_wait<0>();
      ++nf;
      first_tile = false;
    }
}

// The TMA form of k_phase_grad as a producer/consumer pipeline.  Warp 8
// produces: per cell tile the F box, per (rho, tau) sub-problem a G box into
// one of kGrStages stages (TMA copies; lane 0 also writes the sub-problem's
// record and arrives).  Warps 0-7 consume in order: the pair of warps 2w, 2w+1
// owns sigma = s0 + w of each round (rows i = 32 (warp & 1) + lane), reduces
// its rows by shuffles and combines the two warps' sums behind an mbarrier of
// the pair alone (both warps arrive and wait, bounded, once per round; the
// partial sums alternate between two buffers), so no block-wide barrier is
// needed; each warp frees a stage with one arrival on its empty barrier.  Same
// sums in the same order as k_phase_grad.
constexpr int kGrStages = 2;

struct GrRec {
  int rho, tau, Ssig, Sups, rem;
};

template <int S>
__global__ void __launch_bounds__(kPcPipeThreads) k_phase_grad_pipe(const __grid_constant__ PcArgs a) {
  using Gm = GradGeom<S, true>;
  constexpr int FP = Gm::FP, GR = Gm::GR, GP = Gm::GP, GB = Gm::GB, NWT = Gm::NWT;
  extern __shared__ __align__(128) float gsm_raw[];
  float* gsm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(gsm_raw) + 127) & ~uintptr_t(127));
  float* F_s = gsm;
  float* G_s = gsm + kGrI * FP;  // [kGrStages][GB]
  __shared__ float part[2][8][S];
  __shared__ GrRec rec[kGrStages];
  __shared__ __align__(8) uint64_t full[kGrStages], empty[kGrStages], ffull, fempty, pbar[4];
  __shared__ int abort_flag;
  const int Nx = a.Nx, Ny = a.Ny, Wx = a.Wx, Wy = a.Wy;
  const int p = blockIdx.x / Ny, q = blockIdx.x % Ny;
  // grid.y = depths x gsplit: part `gpart` of the depth's (rho, tau) sub-problems
  const int gsplit = a.gsplit > 0 ? a.gsplit : 1;
  const int gpart = (int)blockIdx.y % gsplit;
  const PcDepth dd = a.d[blockIdx.y / gsplit];
  const int Ks = dd.Ks, Kt = dd.Kt;
  float* dA = a.out + dd.off + ((long long)p * Ny + q) * Ks * Kt;
  const int nI = (Wx - p + Nx - 1) / Nx, nJ = (Wy - q + Ny - 1) / Ny;
  const int ntile = ((nI + kGrI - 1) / kGrI) * ((nJ + kGrJ - 1) / kGrJ);
  const int nsub_all = min(Nx, Ks) * min(Ny, Kt);
  const int k_lo = (int)((long long)nsub_all * gpart / gsplit);
  const int nsub = (int)((long long)nsub_all * (gpart + 1) / gsplit) - k_lo;  // per tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kGrStages; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 8);
    }
    mbar_init(smem_addr(&ffull), 1);
    mbar_init(smem_addr(&fempty), 8);
    for (int w = 0; w < 4; ++w) mbar_init(smem_addr(&pbar[w]), 2);  // the two warps of a pair
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int njt = (nJ + kGrJ - 1) / kGrJ;

  if (warp == 8) {
    // ---- producer warp (lane 0 issues; the others only take part in the drain)
    int issued = 0, tiles = 0;
    bool ok = true;
    if (lane == 0) {
      for (int tl = 0; tl < ntile && ok; ++tl) {
        const int i0 = (tl / njt) * kGrI, j0 = (tl % njt) * kGrJ;
        if (tl > 0 && !(ok = mbar_wait_bounded(smem_addr(&fempty), (uint32_t)((tl - 1) & 1),
                                               &abort_flag, kPcWaitNs)))
          break;
        fence_proxy_async_smem();
        mbar_expect_tx(smem_addr(&ffull), (uint32_t)(kGrI * FP * sizeof(float)));
        if (!a.fault) tma_load_3d(smem_addr(F_s), &a.tmap, j0, i0, p * Ny + q, smem_addr(&ffull));
        mbar_arrive(smem_addr(&ffull));
        ++tiles;
        PcSub c;
        pc_sub_depth(c, 0, Ks, Kt, p, q, Nx, Ny);
        for (int k = 0; k < k_lo; ++k) pc_sub_next_phase(c, p, q, Nx, Ny);
        for (int k = 0; k < nsub; ++k) {
          const int s = issued % kGrStages;
          if (issued >= kGrStages &&
              !(ok = mbar_wait_bounded(smem_addr(&empty[s]),
                                       (uint32_t)((issued / kGrStages - 1) & 1), &abort_flag,
                                       kPcWaitNs)))
            break;
          rec[s] = GrRec{c.rho, c.tau, c.Ssig, c.Sups, c.qy & 3};
          fence_proxy_async_smem();
          const uint32_t b = smem_addr(&full[s]);
          mbar_expect_tx(b, (uint32_t)(GR * GP * sizeof(float)));
          if (!a.fault)
            tma_load_3d(smem_addr(G_s + s * GB), &a.tmap2, j0 + c.qy - (c.qy & 3), i0 + c.qx,
                        (dd.z * Nx + c.ar) * Ny + c.br, b);
          mbar_arrive(b);  // releases rec[s]
          ++issued;
          pc_sub_next_phase(c, p, q, Nx, Ny);
        }
      }
      if (!ok) {
        abort_flag = 1;
        if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
      }
      // nothing of this CTA may still be landing when it exits (none were
      // issued under the stall injection)
      for (int j = issued - 1; !a.fault && j >= 0 && j >= issued - kGrStages; --j)
        mbar_wait_bounded(smem_addr(&full[j % kGrStages]), (uint32_t)((j / kGrStages) & 1), nullptr,
                          kPcWaitNs);
      if (tiles > 0 && !a.fault)
        mbar_wait_bounded(smem_addr(&ffull), (uint32_t)((tiles - 1) & 1), nullptr, kPcWaitNs);
    }
    return;
  }

  // ---- consumer warps
  const int i = ((warp & 1) << 5) + lane, pair = warp >> 1;
  int used = 0, round = 0;
  for (int tl = 0; tl < ntile; ++tl) {
    if (!mbar_wait_bounded(smem_addr(&ffull), (uint32_t)(tl & 1), &abort_flag, kPcWaitNs)) {
      if (lane == 0) {
        abort_flag = 1;
        if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
      }
      return;
    }
    for (int k = 0; k < nsub; ++k, ++used) {
      const int s = used % kGrStages;
      if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)((used / kGrStages) & 1), &abort_flag,
                             kPcWaitNs)) {
        if (lane == 0) {
          abort_flag = 1;
          if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
        }
        return;
      }
      const GrRec r = rec[s];
      const float* Gb = G_s + s * GB;
      for (int s0 = 0; s0 < S; s0 += 4, ++round) {
        const int sg = s0 + pair;
        float acc[S];
#pragma unroll
        for (int up = 0; up < S; ++up) acc[up] = 0.f;
        if (sg < S) {
          const float* Fr = F_s + i * FP;
          const float* Gr = Gb + (i + sg) * GP;
          switch (r.rem) {
            case 0: grad_row<S, 0, NWT>(Fr, Gr, acc); break;
            case 1: grad_row<S, 1, NWT>(Fr, Gr, acc); break;
            case 2: grad_row<S, 2, NWT>(Fr, Gr, acc); break;
            default: grad_row<S, 3, NWT>(Fr, Gr, acc); break;
          }
        }
        // the warp's 32 rows by a shuffle tree, then the pair's two warps in order
        float* pt = part[round & 1][warp];
#pragma unroll
        for (int up = 0; up < S; ++up) {
          float v = acc[up];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) pt[up] = v;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&pbar[pair]));  // releases pt
        if (!mbar_wait_bounded(smem_addr(&pbar[pair]), (uint32_t)(round & 1), &abort_flag,
                               kPcWaitNs)) {
          if (lane == 0) {
            abort_flag = 1;
            if (a.status) atomicCAS(a.status, 0, kStatusTimeout);
          }
          return;
        }
        if ((warp & 1) == 0 && lane < S && sg < r.Ssig && lane < r.Sups) {
          const float v = part[round & 1][warp][lane] + part[round & 1][warp + 1][lane];
          float* o = dA + (size_t)(Nx * sg + r.rho) * Kt + (Ny * lane + r.tau);
          *o = tl == 0 ? v : *o + v;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&empty[s]));  // this warp is done with stage s
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(&fempty));  // ... and with the tile's F
  }
}

// The same sum for DB depths of one cut-out size that read the same input
// image (the backprojections): each staged subgrid of the shared image feeds
// the DB depths' weights, so staging is paid once per DB depths.  Block: one
// output phase, a 32 x 64 output tile, depths d[blockIdx.y*DB .. +DB) (missing
// depths at the end get zero weights and no output).
template <int S, int DB, bool kTma>
// 3 blocks per SM (at most 85 registers): one RL update 3.85 -> 3.73 ms against 2
// blocks (128 registers) on the same GPU; 4 blocks per SM measured 3.73 against
// 3.63 ms for 3, and a ring of three buffers with one block barrier per
// sub-problem (spills at DB = 4) 3.77 against 3.63 ms.
__global__ void __launch_bounds__(kPcThreads, 3) k_phase_conv_md(const __grid_constant__ PcArgs a) {
  constexpr int RI = 4, TI = 8 * RI;
  constexpr int S4 = (S + 3) & ~3;
  constexpr int IR = TI + S - 1;
  constexpr int RH = RI / 2;
  constexpr int IC = kPcTJ + S + 3;
  constexpr int ICP = kTma ? PcBox<S>::BX : (IC + 3) & ~3;
  constexpr int IB = (IR * ICP + 31) & ~31;  // buffer stride: 128-byte aligned TMA destinations
  __shared__ __align__(16) float w_s[2][DB * S * S4];
  __shared__ __align__(128) float I_s[2][IB];
  __shared__ __align__(8) uint64_t full[2];
  const int Nx = a.Nx, Ny = a.Ny, Wx = a.Wx, Wy = a.Wy;
  int t = blockIdx.x;
  const int tj = t % a.nTJ;
  t /= a.nTJ;
  const int ti = t % a.nTI;
  t /= a.nTI;
  const int py = t % Ny, px = t / Ny;
  const int i0 = ti * TI, j0 = tj * kPcTJ;
  const int tid = threadIdx.x, wi = tid >> 5, lane = tid & 31;
  // lanes 0-15 and 16-31 take the two halves of the warp's RI rows; 4 columns each
  const int a0 = wi * RI + (lane >> 4) * RH, b0 = 4 * (lane & 15);
  const int dbase = (int)blockIdx.y * DB;
  const int nd = min(DB, a.ndepth - dbase);
  const int Ks = a.d[dbase].Ks, Kt = a.d[dbase].Kt;
  static_assert(DB * S * S4 <= kPcThreads, "one weight per thread");
  // this thread's weight slot: depth wd, tap row wsg, column wup (fixed for the block)
  const int wd = tid / (S * S4), wsg = (tid - wd * (S * S4)) / S4, wup = tid % S4;
  const float* wAz = a.A + (wd < nd ? a.d[dbase + wd].off : 0);
  if (kTma) {
    if (tid == 0) {
      mbar_init(smem_addr(&full[0]), 1);
      mbar_init(smem_addr(&full[1]), 1);
      fence_mbar_init();
    }
    __syncthreads();
  }

  auto stage = [&](const PcSub& c, int buf) {
    if (tid < DB * S * S4) {
      const bool ok = wd < nd && wsg < c.Ssig && wup < c.Sups;
      const int u = Nx * wsg + c.rho, v = Ny * wup + c.tau;
      const float* src =
          !ok ? a.A
              : a.mapped ? wAz + (((size_t)c.ar * Ny + c.br) * Ks + (Ks - 1 - u)) * Kt + (Kt - 1 - v)
                         : wAz + (((size_t)px * Ny + py) * Ks + u) * Kt + v;
      cp_async4(&w_s[buf][tid], src, ok);
    }
    if (kTma) {
      if (tid == 0)
        pc_tma_stage(a, c, 0, I_s[buf], &full[buf], i0, j0, (uint32_t)(IR * ICP * sizeof(float)));
    } else {
      pc_stage_input<IR, IC, ICP>(I_s[buf], a.in, a.in, Nx, Ny, Wx, Wy, i0, j0, c.xoff, c.yoff,
                                  wi, lane);
    }
    cp_async_commit();
  };

  float acc[DB][RH][4];
#pragma unroll
  for (int d = 0; d < DB; ++d)
#pragma unroll
    for (int i = 0; i < RH; ++i) acc[d][i][0] = acc[d][i][1] = acc[d][i][2] = acc[d][i][3] = 0.f;
  PcSub cur;
  pc_sub_depth(cur, dbase, Ks, Kt, px, py, Nx, Ny);
  stage(cur, 0);
  for (int k = 0;; ++k) {
    const int buf = k & 1;
    PcSub nxt = cur;
    const bool more = pc_sub_next_phase(nxt, px, py, Nx, Ny);
    if (more)
      stage(nxt, buf ^ 1);
    else
      cp_async_commit();
    cp_async_wait<1>();  // this thread's weights; published by the barrier in pc_abort or below
    if (kTma) {
      const bool ok = mbar_wait_bounded(smem_addr(&full[buf]), (uint32_t)((k >> 1) & 1), nullptr,
                                        kPcWaitNs);
      if (pc_abort(a, !ok)) {
        if (tid == 0 && more)
          mbar_wait_bounded(smem_addr(&full[buf ^ 1]), (uint32_t)(((k + 1) >> 1) & 1), nullptr,
                            kPcWaitNs);
        return;
      }
    } else {
      __syncthreads();
    }
    const float* wbs[DB];
#pragma unroll
    for (int d = 0; d < DB; ++d) wbs[d] = w_s[buf] + d * (S * S4);
    if (kTma)
      pc_products_rem<S, RH, ICP, DB>(cur.qy & 3, I_s[buf], wbs, a0, b0, acc);
    else
      pc_products<S, RH, 0, ICP, DB>(I_s[buf], wbs, a0, b0, acc);
    __syncthreads();
    if (!more) break;
    cur = nxt;
  }
  cp_async_wait<0>();

#pragma unroll
  for (int d = 0; d < DB; ++d) {
    if (d >= nd) break;
    const long long zo = (long long)a.d[dbase + d].z * a.out_zstride;
#pragma unroll
    for (int i = 0; i < RH; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int X = px + Nx * (i0 + a0 + i), Y = py + Ny * (j0 + b0 + c);
        if (X >= Wx || Y >= Wy) continue;
        const long long o = zo + (long long)X * Wy + Y;
        if (a.epi == kEpiStore) {
          a.out[o] = acc[d][i][c];
        } else if (a.epi == kEpiAccumulate) {
          a.out[o] += acc[d][i][c];
        } else {
          const float n = a.norm[o];
          a.out[o] = n != 0.f ? (a.g[o] / n) * acc[d][i][c] : 0.f;
        }
      }
  }
}

// Quotient of Eq. 2 in place: r = f / fe where fe != 0, else 0.
__global__ void k_rl_quotient(const float* __restrict__ f, float* fe_r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float fe = fe_r[i];
    fe_r[i] = fe != 0.f ? f[i] / fe : 0.f;
  }
}

// Sum of per-depth partial forward projections (fixed order z = 0..Nz-1),
// then the quotient of Eq. 2: r[i] = f[i] / sum_z parts[z][i] (0 where the
// sum is 0).
__global__ void k_rl_sum_quotient(const float* __restrict__ parts, int Nz, long long n,
                                  const float* __restrict__ f, float* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < Nz; ++z) s += parts[(long long)z * n + i];
    r[i] = s != 0.f ? f[i] / s : 0.f;
  }
}

__global__ void k_fill(float* x, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

// Block: one cell position (p, q) of one depth; threads own output taps
// e = (u, v).  The pixels of that cell, f(p + Nx i, q + Ny j), are staged in
// shared memory (in row chunks) and broadcast; dL/dg is read with consecutive
// v on consecutive threads.
constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads)
    k_backproject_grad(const float* __restrict__ f, const float* __restrict__ dg, int Nx, int Ny,
                       int Ks, int Kt, int Wx, int Wy, float* __restrict__ dA, int rows_per_chunk) {
  extern __shared__ float fs[];  // [rows_per_chunk][nJ]
  const int p = blockIdx.x / Ny, q = blockIdx.x % Ny;
  const int cs = (Ks - 1) / 2, ct = (Kt - 1) / 2;
  const int nI = (Wx - p + Nx - 1) / Nx, nJ = (Wy - q + Ny - 1) / Ny;  // pixels of cell (p, q)
  const int KK = Ks * Kt;
  float* out = dA + ((size_t)p * Ny + q) * KK;
  for (int e0 = blockIdx.y * kGradThreads; e0 < KK; e0 += gridDim.y * kGradThreads) {
    const int e = e0 + threadIdx.x;
    const bool active = e < KK;
    const int u = active ? e / Kt : 0, v = active ? e - (e / Kt) * Kt : 0;
    float acc = 0.f;
    for (int i0 = 0; i0 < nI; i0 += rows_per_chunk) {
      const int ni = min(rows_per_chunk, nI - i0);
      __syncthreads();
      for (int k = threadIdx.x; k < ni * nJ; k += kGradThreads) {
        const int di = k / nJ, jj = k - di * nJ;
        fs[k] = __ldg(f + (size_t)(p + Nx * (i0 + di)) * Wy + (q + Ny * jj));
      }
      __syncthreads();
      if (!active) continue;
      for (int di = 0; di < ni; ++di) {
        const int Xv = p + Nx * (i0 + di) + u - cs;  // voxel row
        if (Xv < 0 || Xv >= Wx) continue;
        const float* grow = dg + (size_t)Xv * Wy;
        const float* frow = fs + di * nJ;
        // voxel column q + Ny j + v - ct must lie in [0, Wy)
        int j_lo = 0, j_hi = nJ - 1;
        const int y0 = q + v - ct;
        if (y0 < 0) j_lo = (-y0 + Ny - 1) / Ny;
        if (y0 + Ny * j_hi >= Wy) j_hi = (Wy - 1 - y0) >= 0 ? (Wy - 1 - y0) / Ny : -1;
        for (int jj = j_lo; jj <= j_hi; ++jj) acc = fmaf(frow[jj], __ldg(grow + y0 + Ny * jj), acc);
      }
    }
    if (active) out[(size_t)u * Kt + v] = acc;
  }
}

}  // namespace lfbp

// ------------------------------------------------------------------ host
namespace lfbp {

int launch_projector(int out_cell, int epi, const float* A, int Nx, int Ny, int Ks, int Kt,
                     const float* in, int Wx, int Wy, float* out, const float* g,
                     const float* norm, cudaStream_t st) {
  const int nI = ((Wx + Nx - 1) / Nx + kSvTI - 1) / kSvTI;
  const int nJ = ((Wy + Ny - 1) / Ny + kSvTJ - 1) / kSvTJ;
  const long long blocks = (long long)Nx * Ny * nI * nJ;
  if (blocks > 0x7fffffffLL) return -1;
  const size_t smem = sizeof(float) * kSvUC * Kt;
  if (smem > 48 * 1024) return -1;
  const dim3 grid((unsigned)blocks), block(kSvTJ, kSvTI);
  if (out_cell) {
    if (epi == kEpiStore)
      k_shift_variant_sum<true, kEpiStore><<<grid, block, smem, st>>>(A, Nx, Ny, Ks, Kt, in, Wx, Wy,
                                                                     out, g, norm, nI, nJ);
    else if (epi == kEpiAccumulate)
      k_shift_variant_sum<true, kEpiAccumulate><<<grid, block, smem, st>>>(
          A, Nx, Ny, Ks, Kt, in, Wx, Wy, out, g, norm, nI, nJ);
    else
      k_shift_variant_sum<true, kEpiRL><<<grid, block, smem, st>>>(A, Nx, Ny, Ks, Kt, in, Wx, Wy,
                                                                  out, g, norm, nI, nJ);
  } else {
    if (epi == kEpiStore)
      k_shift_variant_sum<false, kEpiStore><<<grid, block, smem, st>>>(A, Nx, Ny, Ks, Kt, in, Wx,
                                                                      Wy, out, g, norm, nI, nJ);
    else if (epi == kEpiAccumulate)
      k_shift_variant_sum<false, kEpiAccumulate><<<grid, block, smem, st>>>(
          A, Nx, Ny, Ks, Kt, in, Wx, Wy, out, g, norm, nI, nJ);
    else
      k_shift_variant_sum<false, kEpiRL><<<grid, block, smem, st>>>(A, Nx, Ny, Ks, Kt, in, Wx, Wy,
                                                                   out, g, norm, nI, nJ);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}


namespace {
constexpr int kPcSizes[] = {3, 5, 7, 9, 11, 13, 15};  // kernel instances (sub-kernel extent S)

constexpr int kPcTmaMaxS = 9;  // TMA path instances: S <= 9 (larger cut-outs are rare)

// Phase planes of the TMA path (see TMA staging above): block = one plane row
// (z, rx, ry, i); threads along j.  Writes are coalesced; the reads, Ny apart,
// come from L2.
__global__ void k_phase_planes(const float* __restrict__ in, long long in_zstride, int Nx, int Ny,
                               int Wx, int Wy, int Pi, int Pjp, float* __restrict__ planes) {
  int t = blockIdx.x;
  const int i = t % Pi;
  t /= Pi;
  const int ry = t % Ny;
  t /= Ny;
  const int rx = t % Nx;
  const int z = t / Nx;
  const int x = Nx * i + rx;
  const float* row = in + (long long)z * in_zstride + (long long)(x < Wx ? x : 0) * Wy;
  float* out = planes + (long long)blockIdx.x * Pjp;
  for (int j = threadIdx.x; j < Pjp; j += blockDim.x) {
    const int y = Ny * j + ry;
    out[j] = (x < Wx && y < Wy) ? __ldg(row + y) : 0.f;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The library's own stream-ordered memory pool on the current device (memory
// is kept across calls: release threshold at the maximum), so that the
// scratch planes of a call cost no device-wide synchronisation and leave the
// application's pools alone.
cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

// Phase planes of one projection input on the stream (stream-ordered
// allocation; release with planes_release).
struct Planes {
  float* ptr = nullptr;
  int Pi = 0, Pjp = 0, nplanes = 0;
};

// LFBP_FAULT=stall: the TMA-path kernels register their copies' bytes without
// issuing them, so every wait on those copies runs out (tests of the timeout
// path; the cp.async path is not affected).
// Helper streams for independent launches of one projection (per device,
// created on first use and kept): launches that write different output
// depths run side by side, so that small ones (a few depths of one cut-out
// size) share the GPU instead of running one after the other.
constexpr int kSideStreams = 4;
struct SideStreams {
  int dev = -1;
  std::mutex mu;  // held from the fork to the join of one projection
  cudaStream_t s[kSideStreams] = {};
  cudaEvent_t fork = nullptr, join[kSideStreams] = {};
};
std::mutex g_side_mu;
std::vector<SideStreams*> g_side;  // never freed: the streams live as long as the process

SideStreams* side_streams() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_side_mu);
  for (SideStreams* s : g_side)
    if (s->dev == dev) return s;
  SideStreams* s = new SideStreams();
  s->dev = dev;
  bool ok = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < kSideStreams; ++i)
    ok = cudaStreamCreateWithFlags(&s->s[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) return nullptr;  // (a partly created set is dropped; launches stay on the caller's stream)
  g_side.push_back(s);
  return s;
}

int stall_injected() {
  const char* s = std::getenv("LFBP_FAULT");
  return s && !std::strcmp(s, "stall");
}

bool pipe_enabled() {
  const char* s = std::getenv("LFBP_PROJ_PIPE");
  return !(s && s[0] == '0');
}

bool tma_enabled() {
  const char* s = std::getenv("LFBP_PROJ_TMA");
  return !(s && s[0] == '0') && encode_tiled() != nullptr;
}

int planes_build(Planes& pl, const float* in, long long in_zstride, int nz, int Nx, int Ny, int Wx,
                 int Wy, cudaStream_t st) {
  pl.Pi = (Wx + Nx - 1) / Nx;
  pl.Pjp = (((Wy + Ny - 1) / Ny) + 3) & ~3;
  const long long rows = (long long)nz * Nx * Ny * pl.Pi;
  if (rows > 0x7fffffffLL || (long long)nz * Nx * Ny > 0x7fffffffLL) return -1;
  pl.nplanes = nz * Nx * Ny;
  cudaMemPool_t pool = scratch_pool();
  if (!pool || cudaMallocFromPoolAsync((void**)&pl.ptr, (size_t)rows * pl.Pjp * sizeof(float), pool,
                                       st) != cudaSuccess) {
    pl.ptr = nullptr;
    return -1;
  }
  k_phase_planes<<<(unsigned)rows, 128, 0, st>>>(in, in_zstride, Nx, Ny, Wx, Wy, pl.Pi, pl.Pjp,
                                                 pl.ptr);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

void planes_release(Planes& pl, cudaStream_t st) {
  if (pl.ptr) cudaFreeAsync(pl.ptr, st);
  pl.ptr = nullptr;
}

// Tensor map over the planes with a box of BX columns x IR rows x 1 plane.
int planes_map(const Planes& pl, int BX, int IR, CUtensorMap* map) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return -1;
  const cuuint64_t dims[3] = {(cuuint64_t)pl.Pjp, (cuuint64_t)pl.Pi, (cuuint64_t)pl.nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)pl.Pjp * sizeof(float),
                                 (cuuint64_t)pl.Pjp * pl.Pi * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)BX, (cuuint32_t)IR, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, pl.ptr, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
             ? 0
             : -1;
}

template <int S, int RI>
int launch_pc_ri(PcArgs& a, const Planes* pl, int ny, cudaStream_t st) {
  // output tiles of 8*RI rows x kPcTJ columns per phase
  a.nTI = ((a.Wx + a.Nx - 1) / a.Nx + 8 * RI - 1) / (8 * RI);
  a.nTJ = ((a.Wy + a.Ny - 1) / a.Ny + kPcTJ - 1) / kPcTJ;
  const long long nblocks = (long long)a.Nx * a.Ny * a.nTI * a.nTJ;
  if (nblocks > 0x7fffffffLL) return -1;
  const dim3 grid((unsigned)nblocks, (unsigned)ny);
  if (S <= kPcTmaMaxS && pl) {
    if (planes_map(*pl, PcBox<S>::BX, 8 * RI + S - 1, &a.tmap)) return -6;
    if (pipe_enabled())  // eight output rows per thread: two stages fit the static limit
      k_phase_conv_pipe<(S <= kPcTmaMaxS ? S : 3), RI, 1, (RI >= 8 ? 2 : kPcStages)>
          <<<grid, kPcPipeThreads, 0, st>>>(a);
    else
      k_phase_conv<S, RI, (S <= kPcTmaMaxS)><<<grid, kPcThreads, 0, st>>>(a);
  } else {
    k_phase_conv<S, RI, false><<<grid, kPcThreads, 0, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

template <int S>
int launch_pc(PcArgs& a, const Planes* pl, int ny, cudaStream_t st) {
  // depth sums run one block per output tile: half-height tiles for more
  // blocks; one depth per block: tall tiles up to S = 9 (more products per
  // staged sub-problem for each thread; measured: 2 rows per thread 5.29 ms,
  // 4 rows 4.50 ms, 8 rows 4.30 ms for the RL update of the autograd workload)
  if (a.sum_depths) return launch_pc_ri<S, 2>(a, pl, ny, st);
  if constexpr (S <= kPcTmaMaxS)
    return launch_pc_ri<S, 8>(a, pl, ny, st);
  else
    return launch_pc_ri<S, 4>(a, pl, ny, st);
}

int launch_pc_size(int S, PcArgs& a, const Planes* pl, int ny, cudaStream_t st) {
  switch (S) {
    case 3: return launch_pc<3>(a, pl, ny, st);
    case 5: return launch_pc<5>(a, pl, ny, st);
    case 7: return launch_pc<7>(a, pl, ny, st);
    case 9: return launch_pc<9>(a, pl, ny, st);
    case 11: return launch_pc<11>(a, pl, ny, st);
    case 13: return launch_pc<13>(a, pl, ny, st);
    default: return launch_pc<15>(a, pl, ny, st);
  }
}

constexpr int kPcDB = 4;  // most depths per block of k_phase_conv_md

// Depths per block for a group of n depths: the fewest idle depth slots
// (ceil(n/DB)*DB - n), ties to the larger DB.  Idle slots cost full FMAs.
// (On the 21-depth differentiation workload, groups of 6, 6 and 7: one RL
// update 3.63 ms by this rule, 3.67 / 3.75 / 4.10 ms with 3 / 2 / 4 depths per
// block throughout.)
int md_depths_per_block(int n) {
  int best = kPcDB, waste = (n + kPcDB - 1) / kPcDB * kPcDB - n;
  for (int db = kPcDB - 1; db >= 2; --db) {
    const int w = (n + db - 1) / db * db - n;
    if (w < waste) {
      waste = w;
      best = db;
    }
  }
  return best;
}

template <int S, int DB>
int launch_md(PcArgs& a, const Planes* pl, dim3 grid, cudaStream_t st) {
  if (pl) {
    // (the pipelined form, k_phase_conv_pipe<S, 4, kPcDB>, measured slower here:
    // 96 registers x 288 threads leave two blocks per SM, like this one)
    if (planes_map(*pl, PcBox<S>::BX, 32 + S - 1, &a.tmap)) return -6;
    k_phase_conv_md<S, DB, true><<<grid, kPcThreads, 0, st>>>(a);
  } else {
    k_phase_conv_md<S, DB, false><<<grid, kPcThreads, 0, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

template <int S>
int launch_md_db(int db, PcArgs& a, const Planes* pl, dim3 grid, cudaStream_t st) {
  switch (db) {
    case 2: return launch_md<S, 2>(a, pl, grid, st);
    case 3: return launch_md<S, 3>(a, pl, grid, st);
    default: return launch_md<S, kPcDB>(a, pl, grid, st);
  }
}

int launch_pc_md(int S, int db, PcArgs& a, const Planes* pl, int ny, cudaStream_t st) {
  // output tiles of 32 rows x kPcTJ columns per phase
  a.nTI = ((a.Wx + a.Nx - 1) / a.Nx + 31) / 32;
  a.nTJ = ((a.Wy + a.Ny - 1) / a.Ny + kPcTJ - 1) / kPcTJ;
  const long long nblocks = (long long)a.Nx * a.Ny * a.nTI * a.nTJ;
  if (nblocks > 0x7fffffffLL) return -1;
  const dim3 grid((unsigned)nblocks, (unsigned)ny);
  switch (S) {  // small cut-outs only: there staging dominates one depth's work
    case 3: return launch_md_db<3>(db, a, pl, grid, st);
    case 5: return launch_md_db<5>(db, a, pl, grid, st);
    default: return launch_md_db<7>(db, a, pl, grid, st);
  }
}
}  // namespace

int phase_conv_size(int Nx, int Ny, int Ks, int Kt) {
  const int s = std::max((Ks + Nx - 1) / Nx, (Kt + Ny - 1) / Ny);
  for (int S : kPcSizes)
    if (s <= S) return S;
  return 0;
}

int launch_phase_projection(const float* A, int mapped, int Nx, int Ny, int Nz,
                            const long long* off, const int* Ks, const int* Kt, const float* in,
                            long long in_zstride, float* out, long long out_zstride,
                            const float* g, const float* norm, int Wx, int Wy, int sum_depths,
                            int epi, int* status, cudaStream_t st) {
  bool any_tma = false;
  for (int z = 0; z < Nz; ++z) {
    const int S = phase_conv_size(Nx, Ny, Ks[z], Kt[z]);
    if (!S) return -1;
    any_tma |= S <= kPcTmaMaxS;
  }
  const int nI = (Wx + Nx - 1) / Nx, nJ = (Wy + Ny - 1) / Ny;
  // the input by phase for the TMA path (released, stream-ordered, on return)
  struct PlanesGuard {
    Planes pl;
    cudaStream_t st;
    ~PlanesGuard() { planes_release(pl, st); }
  } pg;
  pg.st = st;
  bool tma = false;
  if (any_tma && Nz > 0 && tma_enabled()) {
    const int r = planes_build(pg.pl, in, in_zstride, in_zstride ? Nz : 1, Nx, Ny, Wx, Wy, st);
    if (r == -6) return -6;  // the relayout launch failed
    tma = r == 0;            // -1: no scratch memory, the cp.async path instead
  }
  const Planes* pl = tma ? &pg.pl : nullptr;
  PcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.status = status;
  a.fault = stall_injected();
  a.A = A;
  a.in = in;
  a.in_zstride = in_zstride;
  a.out = out;
  a.out_zstride = out_zstride;
  a.g = g;
  a.norm = norm;
  a.Nx = Nx;
  a.Ny = Ny;
  a.Wx = Wx;
  a.Wy = Wy;
  a.mapped = mapped;
  a.sum_depths = sum_depths;
  // (each launcher sets the output tiling of its kernel: nTI, nTJ)
  if ((long long)Nx * Ny * ((nI + 15) / 16) * ((nJ + kPcTJ - 1) / kPcTJ) > 0x7fffffffLL) return -1;
  // Without a sum over depths every launch writes its own output depths: the
  // launches fork from the caller's stream onto helper streams and join it
  // again before the scratch planes are released (stream order).  With a sum,
  // they run in order on the caller's stream (the sum's order is fixed).
  SideStreams* side = sum_depths ? nullptr : side_streams();
  std::unique_lock<std::mutex> side_lock;  // released after the join below
  if (side) side_lock = std::unique_lock<std::mutex>(side->mu);
  int nlaunch = 0;
  bool forked = false;
  auto next_stream = [&]() -> cudaStream_t {
    if (!side) return st;
    if (!forked) {
      if (cudaEventRecord(side->fork, st) != cudaSuccess) return st;
      for (int i = 0; i < kSideStreams; ++i) cudaStreamWaitEvent(side->s[i], side->fork, 0);
      forked = true;
    }
    return side->s[nlaunch++ % kSideStreams];
  };
  struct JoinGuard {
    SideStreams*& side;
    bool& forked;
    cudaStream_t st;
    ~JoinGuard() {
      if (!side || !forked) return;
      for (int i = 0; i < kSideStreams; ++i) {
        cudaEventRecord(side->join[i], side->s[i]);
        cudaStreamWaitEvent(st, side->join[i], 0);
      }
    }
  } jg{side, forked, st};
  // depths that read one shared image (backprojections) in groups of one
  // cut-out size: several depths per block (k_phase_conv_md)
  std::vector<char> done(Nz, 0);
  if (!sum_depths && in_zstride == 0) {
    for (int z0 = 0; z0 < Nz; ++z0) {
      if (done[z0]) continue;
      std::vector<int> grp;
      for (int z = z0; z < Nz; ++z)
        if (!done[z] && Ks[z] == Ks[z0] && Kt[z] == Kt[z0]) grp.push_back(z);
      const int S = phase_conv_size(Nx, Ny, Ks[z0], Kt[z0]);
      if ((int)grp.size() < 3 || S > 7) continue;  // one depth per block
      for (size_t g0 = 0; g0 < grp.size(); g0 += kPcMaxDepths) {
        const int n = (int)std::min(grp.size() - g0, (size_t)kPcMaxDepths);
        for (int i = 0; i < n; ++i) {
          const int z = grp[g0 + i];
          a.d[i].off = off[z];
          a.d[i].Ks = Ks[z];
          a.d[i].Kt = Kt[z];
          a.d[i].z = z;
          done[z] = 1;
        }
        a.ndepth = n;
        a.epi = epi;
        const int db = md_depths_per_block(n);
        const int rc = launch_pc_md(S, db, a, pl, (n + db - 1) / db, next_stream());
        if (rc) return rc;
      }
    }
  }
  bool first = true;
  for (int S : kPcSizes) {  // one launch per instance size (and per 64 depths)
    int n = 0;
    for (int z = 0; z <= Nz; ++z) {
      const bool take = z < Nz && !done[z] && phase_conv_size(Nx, Ny, Ks[z], Kt[z]) == S;
      if (take) {
        a.d[n].off = off[z];
        a.d[n].Ks = Ks[z];
        a.d[n].Kt = Kt[z];
        a.d[n].z = z;
        ++n;
      }
      if (n == kPcMaxDepths || (z == Nz && n > 0)) {
        a.ndepth = n;
        // summed depths: the first launch stores (or applies epi), later ones add
        a.epi = sum_depths ? (first ? epi : kEpiAccumulate) : epi;
        const int rc = launch_pc_size(S, a, pl, sum_depths ? 1 : n, next_stream());
        if (rc) return rc;
        first = false;
        n = 0;
      }
    }
  }
  return 0;
}

namespace {
template <int S, bool kTma>
int launch_grad_t(const PcArgs& a, dim3 grid, cudaStream_t st) {
  // (set at every launch: the attribute belongs to the current device)
  if (cudaFuncSetAttribute(k_phase_grad<S, kTma>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)GradGeom<S, kTma>::smem) != cudaSuccess)
    return -6;
  k_phase_grad<S, kTma><<<grid, 256, GradGeom<S, kTma>::smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

template <int S>
int launch_grad_pipe(const PcArgs& a, dim3 grid, cudaStream_t st) {
  using Gm = GradGeom<S, true>;
  const size_t smem = sizeof(float) * (kGrI * Gm::FP + kGrStages * Gm::GB) + 128;
  if (cudaFuncSetAttribute(k_phase_grad_pipe<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return -6;
  // enough blocks for about three waves at three blocks per SM: the cells of a
  // depth times its depths can be fewer than the GPU holds, so each cell's
  // sub-problems are shared among gsplit blocks (they write disjoint outputs)
  PcArgs b = a;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -6;
  const long long blocks = (long long)grid.x * grid.y;
  b.gsplit = (int)std::min<long long>(8, std::max<long long>(1, (9LL * sms + blocks - 1) / blocks));
  const int nsub_min = [&] {
    int m = 1 << 30;
    for (int i = 0; i < a.ndepth; ++i)
      m = std::min(m, std::min(a.Nx, a.d[i].Ks) * std::min(a.Ny, a.d[i].Kt));
    return m;
  }();
  b.gsplit = std::max(1, std::min(b.gsplit, nsub_min));
  const dim3 g2(grid.x, grid.y * (unsigned)b.gsplit);
  k_phase_grad_pipe<S><<<g2, kPcPipeThreads, smem, st>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

// With phase planes of f (pf) and dg (pg): tensor maps for the F box
// (kGrI rows x FP columns) and the G boxes (GR rows x GP columns).
template <int S>
int launch_grad(PcArgs& a, const Planes* pf, const Planes* pg, dim3 grid, cudaStream_t st) {
  if (S <= kPcTmaMaxS && pf && pg) {
    using Gm = GradGeom<S, true>;
    if (planes_map(*pf, Gm::FP, kGrI, &a.tmap) || planes_map(*pg, Gm::GP, Gm::GR, &a.tmap2))
      return -6;
    if (pipe_enabled()) return launch_grad_pipe<(S <= kPcTmaMaxS ? S : 3)>(a, grid, st);
    return launch_grad_t<S, (S <= kPcTmaMaxS)>(a, grid, st);
  }
  return launch_grad_t<S, false>(a, grid, st);
}
}  // namespace

int launch_phase_grad(const float* f, const float* dg, int Nx, int Ny, int Nz, const long long* off,
                      const int* Ks, const int* Kt, int Wx, int Wy, float* dA, int* status,
                      cudaStream_t st) {
  bool any_tma = false;
  for (int z = 0; z < Nz; ++z) {
    const int S = phase_conv_size(Nx, Ny, Ks[z], Kt[z]);
    if (!S) return -1;
    any_tma |= S <= kPcTmaMaxS;
  }
  if ((long long)Nx * Ny > 0x7fffffffLL) return -1;
  // f and dg by phase for the TMA path (released, stream-ordered, on return)
  struct Guard {
    Planes pf, pg;
    cudaStream_t st;
    ~Guard() {
      planes_release(pf, st);
      planes_release(pg, st);
    }
  } gd;
  gd.st = st;
  bool tma = false;
  if (any_tma && Nz > 0 && tma_enabled()) {
    const int r1 = planes_build(gd.pf, f, 0, 1, Nx, Ny, Wx, Wy, st);
    const int r2 = r1 ? r1 : planes_build(gd.pg, dg, (long long)Wx * Wy, Nz, Nx, Ny, Wx, Wy, st);
    if (r1 == -6 || r2 == -6) return -6;
    tma = r1 == 0 && r2 == 0;
  }
  const Planes* pf = tma ? &gd.pf : nullptr;
  const Planes* pg = tma ? &gd.pg : nullptr;
  PcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.status = status;
  a.fault = stall_injected();
  a.in = f;
  a.g = dg;
  a.out_zstride = (long long)Wx * Wy;
  a.out = dA;
  a.Nx = Nx;
  a.Ny = Ny;
  a.Wx = Wx;
  a.Wy = Wy;
  for (int S : kPcSizes) {
    int n = 0;
    for (int z = 0; z <= Nz; ++z) {
      if (z < Nz && phase_conv_size(Nx, Ny, Ks[z], Kt[z]) == S) {
        a.d[n].off = off[z];
        a.d[n].Ks = Ks[z];
        a.d[n].Kt = Kt[z];
        a.d[n].z = z;
        ++n;
      }
      if (n == kPcMaxDepths || (z == Nz && n > 0)) {
        a.ndepth = n;
        const dim3 grid((unsigned)(Nx * Ny), (unsigned)n);
        int rc = 0;
        switch (S) {
          case 3: rc = launch_grad<3>(a, pf, pg, grid, st); break;
          case 5: rc = launch_grad<5>(a, pf, pg, grid, st); break;
          case 7: rc = launch_grad<7>(a, pf, pg, grid, st); break;
          case 9: rc = launch_grad<9>(a, pf, pg, grid, st); break;
          case 11: rc = launch_grad<11>(a, pf, pg, grid, st); break;
          case 13: rc = launch_grad<13>(a, pf, pg, grid, st); break;
          default: rc = launch_grad<15>(a, pf, pg, grid, st); break;
        }
        if (rc) return rc;
        if (cudaGetLastError() != cudaSuccess) return -6;
        n = 0;
      }
    }
  }
  return 0;
}

static unsigned elementwise_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

int launch_rl_quotient(const float* f, float* fe_r, long long n, cudaStream_t st) {
  k_rl_quotient<<<elementwise_blocks(n), 256, 0, st>>>(f, fe_r, n);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

int launch_rl_sum_quotient(const float* parts, int Nz, long long n, const float* f, float* r,
                           cudaStream_t st) {
  k_rl_sum_quotient<<<elementwise_blocks(n), 256, 0, st>>>(parts, Nz, n, f, r);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

int launch_fill(float* x, long long n, float v, cudaStream_t st) {
  k_fill<<<elementwise_blocks(n), 256, 0, st>>>(x, n, v);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

int launch_backproject_grad(const float* f, const float* dg, int Nx, int Ny, int Ks, int Kt,
                            int Wx, int Wy, float* dA, cudaStream_t st) {
  const int nJ = (Wy + Ny - 1) / Ny;
  int rows = (12 * 1024) / (int)(sizeof(float) * (nJ > 0 ? nJ : 1));
  if (rows < 1) return -1;
  const int KK = Ks * Kt;
  const int ychunks = (KK + kGradThreads - 1) / kGradThreads;
  dim3 grid(Nx * Ny, ychunks > 65535 ? 65535 : ychunks);
  k_backproject_grad<<<grid, kGradThreads, sizeof(float) * rows * nJ, st>>>(f, dg, Nx, Ny, Ks, Kt,
                                                                          Wx, Wy, dA, rows);
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

}  // namespace lfbp
