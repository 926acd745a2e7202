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
#include <cuda_runtime.h>

#include <cstdint>

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

// Quotient of Eq. 2 in place: r = f / fe where fe != 0, else 0.
__global__ void k_rl_quotient(const float* __restrict__ f, float* fe_r, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float fe = fe_r[i];
    fe_r[i] = fe != 0.f ? f[i] / fe : 0.f;
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

int launch_shift_variant_sum(const float* A, int Nx, int Ny, int Ks, int Kt, const float* in,
                             int Wx, int Wy, float* out, int accumulate, cudaStream_t st) {
  return launch_projector(0, accumulate ? kEpiAccumulate : kEpiStore, A, Nx, Ny, Ks, Kt, in, Wx,
                          Wy, out, nullptr, nullptr, st);
}

static unsigned elementwise_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

int launch_rl_quotient(const float* f, float* fe_r, long long n, cudaStream_t st) {
  k_rl_quotient<<<elementwise_blocks(n), 256, 0, st>>>(f, fe_r, n);
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
