// Host launchers of the projector kernels (lfbp_project.cu), shared with the
// C-ABI in lfbp.cu.  All return 0 on success, nonzero on a launch failure or
// a shape the kernels do not take.
#pragma once
#include <cuda_runtime.h>

namespace lfbp {

// Epilogues of the shift-variant sum.
constexpr int kEpiStore = 0;       // out = sum
constexpr int kEpiAccumulate = 1;  // out += sum (the forward sum over depths)
constexpr int kEpiRL = 2;          // out = g / norm * sum, 0 where norm = 0 (Eq. 2)

// out(P) = sum_k in(P-k+c) * A[(P-k+c) mod N][k]   (out_cell = 0: source cell)
// out(P) = sum_k in(P+k-c) * A[P mod N][k]         (out_cell = 1: output cell)
// on a Wx x Wy grid, terms outside the input dropped; g and norm are read at
// the output's index (kEpiRL only; out may equal g).
int launch_projector(int out_cell, int epi, const float* A, int Nx, int Ny, int Ks, int Kt,
                     const float* in, int Wx, int Wy, float* out, const float* g,
                     const float* norm, cudaStream_t st);
// dA[p][q][u][v] = sum over pixels S of cell (p, q) of f[S] * dg[S + (u-c_s, v-c_t)]
int launch_backproject_grad(const float* f, const float* dg, int Nx, int Ny, int Ks, int Kt,
                            int Wx, int Wy, float* dA, cudaStream_t st);
// The output-cell sum out(P) = sum_{u,v} in(P + (u,v) - c) * w_{P mod N}[u][v]
// over the plan's depths, w = A[p][q] (mapped = 0) or the map of A (mapped = 1:
// w_{p,q}[u][v] = A[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]).
// Depth z's pattern starts at A + off[z]; its input image at in + z*in_zstride;
// per-depth outputs at out + z*out_zstride, or, with sum_depths, one output
// summed over depths in order.  Returns -1 (nothing launched) when a depth's
// cut-out exceeds 15 cells per axis; the caller then uses launch_projector.
// `status`: the device status word, where a kernel whose bounded wait ran out
// records LFBP_ERR_TIMEOUT.  Cut-outs of up to 9 cells per axis take the TMA
// path (the input laid out by phase in a stream-ordered scratch buffer, one
// tensor copy per sub-problem) unless LFBP_PROJ_TMA=0.
int launch_phase_projection(const float* A, int mapped, int Nx, int Ny, int Nz,
                            const long long* off, const int* Ks, const int* Kt, const float* in,
                            long long in_zstride, float* out, long long out_zstride,
                            const float* g, const float* norm, int Wx, int Wy, int sum_depths,
                            int epi, int* status, cudaStream_t st);
// dA_z[p][q][u][v] = sum over pixels S of cell (p, q) of f[S] * dg_z[S + (u-c_s, v-c_t)]
// for every depth (dA_z at dA + off[z], dg_z at dg + z*Wx*Wy); -1 (nothing
// launched) when a cut-out exceeds 15 cells per axis (use launch_backproject_grad).
int launch_phase_grad(const float* f, const float* dg, int Nx, int Ny, int Nz, const long long* off,
                      const int* Ks, const int* Kt, int Wx, int Wy, float* dA, int* status,
                      cudaStream_t st);
// fe_r[i] = f[i] / fe_r[i] where fe_r[i] != 0, else 0 (the quotient of Eq. 2)
int launch_rl_quotient(const float* f, float* fe_r, long long n, cudaStream_t st);
// r[i] = f[i] / sum_{z < Nz} parts[z*n + i] (fixed order; 0 where the sum is 0)
int launch_rl_sum_quotient(const float* parts, int Nz, long long n, const float* f, float* r,
                           cudaStream_t st);
int launch_fill(float* x, long long n, float v, cudaStream_t st);

}  // namespace lfbp
