// Index arithmetic of the literal paper-window map (Sec. 4, Eqs. 4-9, Fig. 10)
// for either parity of the cut-out, shared by the CUDA kernel of
// lfbp_window.cu and by a host test harness (compiled as plain C++ there).
#pragma once

#if defined(__CUDACC__)
#define LFBP_WINDOW_FN __host__ __device__ __forceinline__
#else
#define LFBP_WINDOW_FN inline
#endif

namespace lfbp {

LFBP_WINDOW_FN int window_floor_div(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// Eq. 5: alpha wrapped into 1..n
LFBP_WINDOW_FN int window_eq5_wrap(int alpha, int n) {
  return alpha - window_floor_div(alpha - 1, n) * n;
}

// Source (0-based cell position a, returned; cut-out index *s0) of output
// (p, u) on one axis of n cell positions and cut-out size K, or -1 when the
// literal loop never writes it:  s = K - s' + (K mod 2) (Eq. 8 solved for s),
// m = x' - s + n + 2 dS - floor((n - 1) / 2) (Eqs. 4 and 6 solved for m),
// valid for 1 <= s, m <= K; the cell is x(m) of Eq. 5.
LFBP_WINDOW_FN int window_source(int p, int u, int n, int K, int* s0) {
  const int xp = p + 1, sp = u + 1;
  const int s = K - sp + (K & 1);
  if (s < 1 || s > K) return -1;
  const int dS = window_floor_div(K - n, 2);
  const int m = xp - s + n + 2 * dS - (n - 1) / 2;
  if (m < 1 || m > K) return -1;
  *s0 = s - 1;
  return window_eq5_wrap(m - dS, n) - 1;
}

}  // namespace lfbp
