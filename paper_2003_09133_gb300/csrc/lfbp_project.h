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
int launch_shift_variant_sum(const float* A, int Nx, int Ny, int Ks, int Kt, const float* in,
                             int Wx, int Wy, float* out, int accumulate, cudaStream_t st);
// dA[p][q][u][v] = sum over pixels S of cell (p, q) of f[S] * dg[S + (u-c_s, v-c_t)]
int launch_backproject_grad(const float* f, const float* dg, int Nx, int Ny, int Ks, int Kt,
                            int Wx, int Wy, float* dA, cudaStream_t st);
// fe_r[i] = f[i] / fe_r[i] where fe_r[i] != 0, else 0 (the quotient of Eq. 2)
int launch_rl_quotient(const float* f, float* fe_r, long long n, cudaStream_t st);
int launch_fill(float* x, long long n, float v, cudaStream_t st);

}  // namespace lfbp
