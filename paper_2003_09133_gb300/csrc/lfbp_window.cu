// The paper-window map with the literal loop ranges of Sec. 4 (Eqs. 4-9,
// Fig. 10) for cut-outs of either parity.  Odd cut-outs take the tiled kernels
// of lfbp.cu; this file serves the even ones.  Eq. 8 then reads s' = n_s - s,
// which drops s = n_s and never writes s' = n_s, so the map is a partial
// injection rather than a permutation.
//
// Per axis (x with s: n = n_x, K = n_s; 1-based as in the paper), the loop over
// s = 1..K and m = 1..K writes
//     H'(s', x'_m) = H(s, x(m)),   alpha_m = m - dS,   dS = floor((K - n) / 2),
//     x(m) = alpha_m wrapped into 1..n (Eq. 5),
//     x'_m = s - n + alpha_m + floor((n - 1) / 2) - dS      (Eq. 6),
//     s'   = K - s + (K mod 2)                                (Eq. 8),
// keeping 0 < x'_m <= n and s' > 0.  x'_m grows with m, so each output
// (x', s') has at most one source, found by solving for s and then m:
//     s = K - s' + (K mod 2),   m = x' - s + n + 2 dS - floor((n - 1) / 2),
// valid when 1 <= s <= K and 1 <= m <= K.  The forward kernel gathers through
// that inverse (zero where there is no source); the adjoint scatters each
// written output back to its source after zeroing the gradient, so every
// source receives at most one value (the m giving valid x'_m for one s are
// n consecutive values, whose x(m) are distinct).
//
// The forward map runs a row at a time through shared memory when a row's Ny
// source segments fit (k_window_literal_rows: coalesced reads and writes);
// otherwise, and for the adjoint, one thread per element with gathered reads.
#include <cuda_runtime.h>

#include <cstdint>

#include "lfbp_project.h"
#include "lfbp_window.cuh"

namespace lfbp {
namespace {

// out[z][p][q][u][v] = in[z][a][b][s][t] through window_source on both axes,
// 0 where either axis has no source (forward); with kAdjoint the same pairs
// move the other way, in -> out at the source positions (out zeroed first).
template <typename T, bool kAdjoint>
__global__ void k_window_literal(const T* __restrict__ in, T* __restrict__ out, int Nx, int Ny,
                                 int Ks, int Kt, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int v = (int)(r % Kt);
    r /= Kt;
    const int u = (int)(r % Ks);
    r /= Ks;
    const int q = (int)(r % Ny);
    const int p = (int)(r / Ny);
    int s0 = 0, t0 = 0;
    const int a = window_source(p, u, Nx, Ks, &s0);
    const int b = window_source(q, v, Ny, Kt, &t0);
    const bool ok = a >= 0 && b >= 0;
    const long long src = ok ? (((long long)a * Ny + b) * Ks + s0) * Kt + t0 : 0;
    if (kAdjoint) {
      if (ok) out[src] = in[e];
    } else {
      out[e] = ok ? in[src] : T(0);
    }
  }
}

// The forward map a row at a time: block (p, u) loads the Ny source rows
// (a, b = 0..Ny-1, s0) of its output row u, Kt elements each and contiguous in
// H, into shared memory with coalesced reads, then writes the Ny x Kt output
// plane (q, v) of (p, u) with coalesced writes.  Needs Ny * Kt elements of
// shared memory.
template <typename T>
__global__ void k_window_literal_rows(const T* __restrict__ in, T* __restrict__ out, int Nx,
                                      int Ny, int Ks, int Kt) {
  extern __shared__ __align__(16) unsigned char wsm[];
  T* rows = reinterpret_cast<T*>(wsm);
  const int u = (int)(blockIdx.x % Ks), p = (int)(blockIdx.x / Ks);
  int s0 = 0;
  const int a = window_source(p, u, Nx, Ks, &s0);
  const long long plane = (long long)Ny * Kt;
  T* dst = out + ((long long)p * Ny * Ks + u) * Kt;  // element (p, q = 0, u, v = 0)
  if (a < 0) {  // the literal loop writes nothing in this row
    for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
      const int q = (int)(e / Kt), v = (int)(e - (long long)q * Kt);
      dst[(long long)q * Ks * Kt + v] = T(0);
    }
    return;
  }
  for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
    const int b = (int)(e / Kt), t = (int)(e - (long long)b * Kt);
    rows[e] = in[(((long long)a * Ny + b) * Ks + s0) * Kt + t];
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
    const int q = (int)(e / Kt), v = (int)(e - (long long)q * Kt);
    int t0 = 0;
    const int b = window_source(q, v, Ny, Kt, &t0);
    dst[(long long)q * Ks * Kt + v] = b >= 0 ? rows[(long long)b * Kt + t0] : T(0);
  }
}

template <typename T>
int launch_t(const void* in, void* out, int Nx, int Ny, int Ks, int Kt, int adjoint,
             cudaStream_t st) {
  const long long n = (long long)Nx * Ny * Ks * Kt;
  if (n == 0) return 0;
  const long long row_bytes = (long long)Ny * Kt * (long long)sizeof(T);
  if (!adjoint && row_bytes <= 48 * 1024 && (long long)Nx * Ks <= 0x7fffffffLL) {
    k_window_literal_rows<T><<<(unsigned)((long long)Nx * Ks), 256, (size_t)row_bytes, st>>>(
        static_cast<const T*>(in), static_cast<T*>(out), Nx, Ny, Ks, Kt);
    return cudaGetLastError() == cudaSuccess ? 0 : -6;
  }
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (adjoint) {
    if (cudaMemsetAsync(out, 0, (size_t)n * sizeof(T), st) != cudaSuccess) return -6;
    k_window_literal<T, true><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const T*>(in), static_cast<T*>(out), Nx, Ny, Ks, Kt, n);
  } else {
    k_window_literal<T, false><<<(unsigned)blocks, 256, 0, st>>>(
        static_cast<const T*>(in), static_cast<T*>(out), Nx, Ny, Ks, Kt, n);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

}  // namespace

int launch_window_literal(const void* in_depth, void* out_depth, int esize, int Nx, int Ny, int Ks,
                          int Kt, int adjoint, cudaStream_t st) {
  if (esize == 4) return launch_t<uint32_t>(in_depth, out_depth, Nx, Ny, Ks, Kt, adjoint, st);
  if (esize == 2) return launch_t<uint16_t>(in_depth, out_depth, Nx, Ny, Ks, Kt, adjoint, st);
  return -1;
}

}  // namespace lfbp
