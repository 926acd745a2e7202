/*
 * CPU BASELINE for the benchmark -- TEST INFRASTRUCTURE ONLY, not the oracle.
 *
 * The paper's own method on the host cores: H' built from H by the closed-form
 * index relations of Sec. 4 (Eqs. 4-9 solved for the full transpose, 0-based):
 *
 *     H'[p][q][u][v] = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]
 *
 * with c = (K-1)/2, for odd cut-outs.  It is the fair CPU counterpart of the
 * GPU path (the paper's algorithm is a CPU rearrangement, Sec. 4 and Table 1),
 * timed by bench.py beside the brute-force oracle.  The work is split over the
 * host cores with OpenMP by output row (depth z, cell row p, pixel row u):
 * every row reads the Ny source rows (a, b, s) of one cut-out row, Kt
 * elements each, and writes Ny contiguous output runs of Kt elements.  The
 * tests check it against oracle_transpose bit for bit; nothing in the
 * product library uses it.
 *
 * Layout as in lfbp_oracle.c: flat, depth-major, ragged; depth z is row-major
 * [a][b][s][t] with Nx*Ny*Ks[z]*Kt[z] elements.  Elements are moved as raw
 * bytes (esize 2 or 4).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int cpu_rearrange_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* One output row (p, u) of one depth: Ny runs of Kt elements. */
#define ROW_BODY(T)                                                                   \
    do {                                                                              \
        const T* src = (const T*)H + off;                                             \
        T* dst = (T*)Hp + off;                                                        \
        const long a = ((long)p + u - cs % Nx + Nx) % Nx;                             \
        const long s = ks - 1 - u;                                                    \
        for (int q = 0; q < Ny; ++q) {                                                \
            T* run = dst + (((size_t)p * Ny + q) * ks + u) * kt;                      \
            long b = ((long)q - ct % Ny + Ny) % Ny; /* b of column v = 0 */            \
            for (int v = 0; v < kt; ++v) {                                            \
                run[v] = src[(((size_t)a * Ny + b) * ks + s) * kt + (kt - 1 - v)];    \
                if (++b == Ny) b = 0;                                                 \
            }                                                                         \
        }                                                                             \
    } while (0)

int cpu_rearrange(const void* H, void* Hp, int esize, int Nx, int Ny, int Nz, const int* Ks,
                  const int* Kt, int nthreads) {
    if (!H || !Hp || !Ks || !Kt || Nx < 1 || Ny < 1 || Nz < 0) return -1;
    if (esize != 2 && esize != 4) return -1;
    cpu_rearrange_threads(nthreads);
    size_t* offs = (size_t*)malloc(sizeof(size_t) * (size_t)(Nz + 1));
    if (!offs) return -2;
    offs[0] = 0;
    long nrows = 0;
    for (int z = 0; z < Nz; ++z) {
        if (Ks[z] < 1 || Kt[z] < 1 || Ks[z] % 2 == 0 || Kt[z] % 2 == 0) { free(offs); return -1; }
        offs[z + 1] = offs[z] + (size_t)Nx * Ny * (size_t)Ks[z] * Kt[z];
        nrows += (long)Nx * Ks[z];
    }
    /* row r -> (z, p, u): depths in order, rows of a depth p-major */
#pragma omp parallel for schedule(dynamic, 4)
    for (long r = 0; r < nrows; ++r) {
        long rem = r;
        int z = 0;
        while (rem >= (long)Nx * Ks[z]) { rem -= (long)Nx * Ks[z]; ++z; }
        const int ks = Ks[z], kt = Kt[z];
        const int p = (int)(rem / ks), u = (int)(rem % ks);
        const long cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        const size_t off = offs[z];
        if (esize == 4)
            ROW_BODY(uint32_t);
        else
            ROW_BODY(uint16_t);
    }
    free(offs);
    return 0;
}
