// Host harness for the literal paper-window map of lfbp_window.cu: the same
// index arithmetic (lfbp_window.cuh, compiled here as plain C++) applied to a
// whole ragged array, element by element, so that the CPU tests can compare
// it with the oracle's literal evaluation of Eqs. (4)-(9).
#include <cstddef>
#include <cstring>

#include "lfbp_window.cuh"

extern "C" int window_apply(const unsigned char* in, unsigned char* out, int esize, int Nx, int Ny,
                            int Nz, const int* Ks, const int* Kt, int adjoint) {
  size_t off = 0;
  for (int z = 0; z < Nz; ++z) {
    const long long n = (long long)Nx * Ny * Ks[z] * Kt[z];
    const unsigned char* src_base = in + off * esize;
    unsigned char* dst_base = out + off * esize;
    if (adjoint) std::memset(dst_base, 0, (size_t)n * esize);
    for (long long e = 0; e < n; ++e) {
      long long r = e;
      const int v = (int)(r % Kt[z]);
      r /= Kt[z];
      const int u = (int)(r % Ks[z]);
      r /= Ks[z];
      const int q = (int)(r % Ny), p = (int)(r / Ny);
      int s0 = 0, t0 = 0;
      const int a = lfbp::window_source(p, u, Nx, Ks[z], &s0);
      const int b = lfbp::window_source(q, v, Ny, Kt[z], &t0);
      const bool ok = a >= 0 && b >= 0;
      const long long src = ok ? (((long long)a * Ny + b) * Ks[z] + s0) * Kt[z] + t0 : 0;
      if (adjoint) {
        if (ok) std::memcpy(dst_base + src * esize, src_base + e * esize, esize);
      } else if (ok) {
        std::memcpy(dst_base + e * esize, src_base + src * esize, esize);
      } else {
        std::memset(dst_base + e * esize, 0, esize);
      }
    }
    off += (size_t)n;
  }
  return 0;
}
