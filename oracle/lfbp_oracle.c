/*
 * lfbp CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the construction of
 * the light-field backprojection array H' from the PSF array H computes
 * (Eberhart, "Efficient computation of backprojection arrays for 3D light
 * field deconvolution", arXiv 2003.09133).  It exists to check the CUDA path:
 * only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Array layout (both H and H'): flat, depth-major, ragged in depth; depth z
 * holds Nx*Ny*Ks[z]*Kt[z] elements in row-major [a][b][s][t] order.  For H,
 * (a, b) is the source (voxel) position inside the elementary cell -- the
 * paper's (x, y) dimensions -- and (s, t) the pixel inside the voxel-centred
 * cut-out.  For H', (a, b) is the pixel position inside the lenslet -- the
 * paper's (x', y') -- and (s, t) the voxel inside the pixel-centred window,
 * the paper's (s', t'): the two arrays have the same shape, with the roles
 * of the cell and pixel dimensions exchanged (Sec. 3, Fig. 6).  The paper's x
 * pairs with s and y with t.
 *
 * Functions and the passage each follows:
 *   oracle_transpose        H' as the transpose of the measurement operator of
 *                           Eq. (1) (Sec. 2.1 forward model; Sec. 3: H'
 *                           collects, per sensor pixel, the weights of the
 *                           voxels that reach it).
 *   oracle_transpose_adjoint  the adjoint (scatter) of that permutation.
 *   oracle_paper_window     Eqs. (4)-(9) evaluated in the paper's 1-based
 *                           notation and loop ranges (Sec. 4), source by
 *                           source.
 *   oracle_forward_f64      f = H g, Eq. (1): copies of the cut-outs of H,
 *                           scaled by the voxel values, summed on the sensor.
 *   oracle_backproject_f64  g = H' f, the backprojection used in Eq. (2).
 *   oracle_backproject_points  the same, one voxel at a time.
 *   oracle_grad_hp_f64      d/dH' of sum (H' f - g_ref)^2 given the residual.
 *   oracle_grad_hp_points   the same, one entry at a time.
 *
 * Parity: every function is pinned by the oracle's own CPU tests against
 * something other than itself (a dense measurement matrix built by pattern
 * placement and transposed with numpy, a hand evaluation of Eqs. (4)-(9),
 * the adjoint identity, closed special cases, central finite differences).
 *
 * Values are moved as raw bytes in the two permutation functions, so NaN
 * payloads, signed zeros, infinities and subnormals survive unchanged.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* floor division and floor modulo for a positive divisor */
static long floor_div(long a, long b) {
    long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}
static long ceil_div(long a, long b) { return -floor_div(-a, b); }
static long floor_mod(long a, long b) { return a - floor_div(a, b) * b; }

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* number of worker threads the OpenMP runtime will use */
int oracle_threads(int nthreads) { return set_threads(nthreads); }

static size_t depth_elems(int Nx, int Ny, int ks, int kt) {
    return (size_t)Nx * (size_t)Ny * (size_t)ks * (size_t)kt;
}

/* ------------------------------------------------------------------------ */
/* Forward-model weight, Eq. (1) with the cut-out convention of Sec. 2.1.    */
/*                                                                          */
/* Voxel X (lateral position in pixel units) emits the pattern stored in    */
/* H[X mod N], whose cut-out bounds move with the voxel ("the bounds of the */
/* cutouts ... must be shifted likewise"): entry k of the cut-out, k in     */
/* [0, K), is recorded by sensor pixel X + k - c with c = (K-1)/2.  So the  */
/* weight of voxel X on pixel S sits at cut-out index k = S - X + c, and is */
/* zero when that index falls outside the cut-out.  The same rule is        */
/* applied independently along each lateral axis.                           */
/* ------------------------------------------------------------------------ */
static int cutout_index(long S, long X, int K) {
    long k = S - X + (K - 1) / 2;
    return (k >= 0 && k < K) ? (int)k : -1;
}

/*
 * H' = transpose of the measurement operator, stored pixel-centred.
 *
 * H'[p][q][u][v] is the weight that voxel X = S + (u - c_s, v - c_t) has on
 * pixel S, for a pixel S whose position inside its lenslet is (p, q).  By the
 * periodicity of the lenslet grid (Sec. 2.1, elementary cell) any such pixel
 * gives the same weight; the pixel of lenslet 0, S = (p, q), is used.  This
 * is the backprojection of a unit image at that pixel through every cut-out
 * of H (Sec. 3, the recipe of the earlier codes), read back on the window of
 * voxels the pixel can see.
 */
int oracle_transpose(const void* H, void* Hp, int esize, int Nx, int Ny, int Nz,
                     const int* Ks, const int* Kt, int nthreads) {
    if (!H || !Hp || !Ks || !Kt || Nx < 1 || Ny < 1 || Nz < 0) return -1;
    if (esize != 1 && esize != 2 && esize != 4 && esize != 8) return -1;
    set_threads(nthreads);
    size_t* off = (size_t*)malloc(sizeof(size_t) * (size_t)(Nz + 1));
    if (!off) return -2;
    off[0] = 0;
    for (int z = 0; z < Nz; ++z) {
        if (Ks[z] < 1 || Kt[z] < 1 || Ks[z] % 2 == 0 || Kt[z] % 2 == 0) { free(off); return -1; }
        off[z + 1] = off[z] + depth_elems(Nx, Ny, Ks[z], Kt[z]);
    }
    const char* src = (const char*)H;
    char* dst = (char*)Hp;
    int bad = 0;
    long nwork = (long)Nz * Nx;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (long w = 0; w < nwork; ++w) {
        int z = (int)(w / Nx), p = (int)(w % Nx);
        int ks = Ks[z], kt = Kt[z];
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        for (int q = 0; q < Ny; ++q)
            for (int u = 0; u < ks; ++u)
                for (int v = 0; v < kt; ++v) {
                    long Sx = p, Sy = q;                 /* the pixel            */
                    long Xx = Sx + u - cs, Xy = Sy + v - ct; /* voxel in its window */
                    int a = (int)floor_mod(Xx, Nx);      /* voxel's cell position */
                    int b = (int)floor_mod(Xy, Ny);
                    int s = cutout_index(Sx, Xx, ks);    /* where X records S     */
                    int t = cutout_index(Sy, Xy, kt);
                    if (s < 0 || t < 0) { bad = 1; continue; }
                    size_t i_in = off[z] + (((size_t)a * Ny + b) * ks + s) * kt + t;
                    size_t i_out = off[z] + (((size_t)p * Ny + q) * ks + u) * kt + v;
                    memcpy(dst + i_out * esize, src + i_in * esize, (size_t)esize);
                }
    }
    free(off);
    return bad ? -3 : 0;
}

/*
 * Adjoint of oracle_transpose as a linear map on arrays: every output element
 * of the transpose is a copy of one input element, so the adjoint scatters
 * each element of dHp back to the H position it was copied from.  Used for
 * the gradient with respect to H of a loss on H' (Sec. 4 notes the mapping
 * is reversible, which the tests check separately).
 */
int oracle_transpose_adjoint(const void* dHp, void* dH, int esize, int Nx, int Ny, int Nz,
                             const int* Ks, const int* Kt, int nthreads) {
    if (!dH || !dHp || !Ks || !Kt || Nx < 1 || Ny < 1 || Nz < 0) return -1;
    if (esize != 1 && esize != 2 && esize != 4 && esize != 8) return -1;
    set_threads(nthreads);
    size_t off = 0;
    const char* src = (const char*)dHp;
    char* dst = (char*)dH;
    int bad = 0;
    for (int z = 0; z < Nz; ++z) {
        int ks = Ks[z], kt = Kt[z];
        if (ks < 1 || kt < 1 || ks % 2 == 0 || kt % 2 == 0) return -1;
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int p = 0; p < Nx; ++p)
            for (int q = 0; q < Ny; ++q)
                for (int u = 0; u < ks; ++u)
                    for (int v = 0; v < kt; ++v) {
                        long Xx = (long)p + u - cs, Xy = (long)q + v - ct;
                        int a = (int)floor_mod(Xx, Nx), b = (int)floor_mod(Xy, Ny);
                        int s = cutout_index(p, Xx, ks), t = cutout_index(q, Xy, kt);
                        if (s < 0 || t < 0) { bad = 1; continue; }
                        size_t i_h = off + (((size_t)a * Ny + b) * ks + s) * kt + t;
                        size_t i_hp = off + (((size_t)p * Ny + q) * ks + u) * kt + v;
                        memcpy(dst + i_h * esize, src + i_hp * esize, (size_t)esize);
                    }
        off += depth_elems(Nx, Ny, ks, kt);
    }
    return bad ? -3 : 0;
}

/*
 * Eqs. (4)-(9) in the paper's 1-based notation, with the paper's loop ranges
 * (its m = 1..n_s and n = 1..n_t) and validity conditions (0 < x' <= n_x,
 * 0 < s'), read from the source side: for every element H(s, t, x, y) the
 * equations give the H' position it is assigned to, or none.
 *
 * One axis (x with s; y with t is the same with n_y, n_t):
 *   Eq. (4):  alpha = m - floor((n_s - n_x)/2)      for a loop index m
 *   Eq. (5):  x(alpha) = alpha wrapped into 1..n_x  (the cell alpha lands in)
 *   Eq. (6):  x' = s - n_x + alpha + floor((n_x-1)/2) - floor((n_s-n_x)/2)
 *   Eq. (8):  s' = n_s - s + (n_s mod 2)
 * Source (x, s) is assigned to (x', s') for the m in 1..n_s whose wrapped
 * alpha is x and whose x' is in 1..n_x, provided s' > 0.  The m with the
 * same x(alpha) differ by n_x, so their x' differ by n_x and at most one of
 * them is valid: every source has at most one target per axis.  The element
 * moves when both axes give a target; H' positions that no source reaches
 * stay zero, and a position reached twice is reported (-3).
 * Even n_s or n_t are accepted here exactly as the equations read.
 */
static long eq5_wrap(long alpha, long n) {
    if (alpha > n) return alpha - floor_div(alpha - 1, n) * n;
    if (alpha <= 0) return alpha + ceil_div(1 - alpha, n) * n;
    return alpha;
}

/* The target (x', s') of source (x, s) on one axis (n cells, cut-out K):
 * returns x' (and *sp = s'), or 0 when the equations assign it nowhere. */
static long axis_target(long x, long s, long n, long K, long* sp) {
    *sp = K - s + (K % 2);
    if (*sp <= 0) return 0;
    long dS = floor_div(K - n, 2);
    for (long m = 1; m <= K; ++m) {
        long alpha = m - dS;
        if (eq5_wrap(alpha, n) != x) continue;
        long xp = s - n + alpha + floor_div(n - 1, 2) - dS;
        if (xp >= 1 && xp <= n) return xp;
    }
    return 0;
}

int oracle_paper_window(const void* H, void* Hp, int esize, int Nx, int Ny, int Nz,
                        const int* Ks, const int* Kt) {
    if (!H || !Hp || !Ks || !Kt || Nx < 1 || Ny < 1 || Nz < 0) return -1;
    if (esize != 1 && esize != 2 && esize != 4 && esize != 8) return -1;
    const char* src = (const char*)H;
    char* dst = (char*)Hp;
    size_t off = 0;
    int twice = 0;
    for (int z = 0; z < Nz; ++z) {
        long ns = Ks[z], nt = Kt[z];
        if (ns < 1 || nt < 1) return -1;
        size_t n = depth_elems(Nx, Ny, (int)ns, (int)nt);
        memset(dst + off * esize, 0, n * (size_t)esize);
        /* per-axis targets of every source, tabulated: [x-1][s-1] -> x', s' */
        long* tx = (long*)malloc(sizeof(long) * (size_t)(Nx * ns));
        long* ts = (long*)malloc(sizeof(long) * (size_t)(Nx * ns));
        long* ty = (long*)malloc(sizeof(long) * (size_t)(Ny * nt));
        long* tt = (long*)malloc(sizeof(long) * (size_t)(Ny * nt));
        unsigned char* hit = (unsigned char*)calloc(n, 1);
        if (!tx || !ts || !ty || !tt || !hit) {
            free(tx); free(ts); free(ty); free(tt); free(hit);
            return -2;
        }
        for (long x = 1; x <= Nx; ++x)
            for (long s = 1; s <= ns; ++s)
                tx[(x - 1) * ns + (s - 1)] = axis_target(x, s, Nx, ns, &ts[(x - 1) * ns + (s - 1)]);
        for (long y = 1; y <= Ny; ++y)
            for (long t = 1; t <= nt; ++t)
                ty[(y - 1) * nt + (t - 1)] = axis_target(y, t, Ny, nt, &tt[(y - 1) * nt + (t - 1)]);
        /* H(s, t, x, y) lives at [x-1][y-1][s-1][t-1]; so does H'(s', t', x', y') */
        for (long x = 1; x <= Nx; ++x)
            for (long y = 1; y <= Ny; ++y)
                for (long s = 1; s <= ns; ++s) {
                    long xp = tx[(x - 1) * ns + (s - 1)], sp = ts[(x - 1) * ns + (s - 1)];
                    if (xp == 0) continue;
                    for (long t = 1; t <= nt; ++t) {
                        long yp = ty[(y - 1) * nt + (t - 1)], tp = tt[(y - 1) * nt + (t - 1)];
                        if (yp == 0) continue;
                        size_t i_in = ((((size_t)(x - 1)) * Ny + (size_t)(y - 1)) * ns
                                       + (size_t)(s - 1)) * nt + (size_t)(t - 1);
                        size_t i_out = ((((size_t)(xp - 1)) * Ny + (size_t)(yp - 1)) * ns
                                        + (size_t)(sp - 1)) * nt + (size_t)(tp - 1);
                        twice |= hit[i_out];
                        hit[i_out] = 1;
                        memcpy(dst + (off + i_out) * esize, src + (off + i_in) * esize,
                               (size_t)esize);
                    }
                }
        free(tx); free(ts); free(ty); free(tt); free(hit);
        off += n;
    }
    return twice ? -3 : 0;
}

/* ------------------------------------------------------------------------ */
/* Projectors on a finite W_x x W_y sensor and a W_x x W_y x Nz volume, in   */
/* FP64.  Voxel grid = pixel grid laterally (Sec. 2.1: lateral voxel sizes   */
/* are tied to the pixel pitch); the cell position of voxel X is X mod N.    */
/* Everything outside the sensor / volume is zero.  H, H' are FP64 arrays in */
/* the layout above; g is [Nz][W_x][W_y], f is [W_x][W_y].                   */
/* ------------------------------------------------------------------------ */

/* f = H g (Eq. 1): each voxel adds its cut-out, scaled by its value, onto the
 * sensor at the pixels the cut-out covers (Sec. 2.1 image formation). */
int oracle_forward_f64(const double* H, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
                       const double* g, int Wx, int Wy, double* f) {
    if (!H || !g || !f || !Ks || !Kt) return -1;
    memset(f, 0, sizeof(double) * (size_t)Wx * (size_t)Wy);
    size_t off = 0;
    for (int z = 0; z < Nz; ++z) {
        int ks = Ks[z], kt = Kt[z];
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        for (long X = 0; X < Wx; ++X)
            for (long Y = 0; Y < Wy; ++Y) {
                double gv = g[((size_t)z * Wx + X) * Wy + Y];
                if (gv == 0.0) continue;
                int a = (int)(X % Nx), b = (int)(Y % Ny);
                const double* pat = H + off + ((size_t)a * Ny + b) * ks * kt;
                for (int s = 0; s < ks; ++s) {
                    long Sx = X + s - cs;                 /* pixel of entry s */
                    if (Sx < 0 || Sx >= Wx) continue;
                    for (int t = 0; t < kt; ++t) {
                        long Sy = Y + t - ct;
                        if (Sy < 0 || Sy >= Wy) continue;
                        f[(size_t)Sx * Wy + Sy] += gv * pat[(size_t)s * kt + t];
                    }
                }
            }
        off += depth_elems(Nx, Ny, ks, kt);
    }
    return 0;
}

/* g = H' f: each pixel S sends its value back into the voxels of its window,
 * weighted by the slice H'[S mod N] (the backprojection inside Eq. 2). */
int oracle_backproject_f64(const double* Hp, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
                           const double* f, int Wx, int Wy, double* g) {
    if (!Hp || !g || !f || !Ks || !Kt) return -1;
    size_t off = 0;
    for (int z = 0; z < Nz; ++z) {
        int ks = Ks[z], kt = Kt[z];
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        double* gz = g + (size_t)z * Wx * Wy;
        memset(gz, 0, sizeof(double) * (size_t)Wx * (size_t)Wy);
        for (long Sx = 0; Sx < Wx; ++Sx)
            for (long Sy = 0; Sy < Wy; ++Sy) {
                double fv = f[(size_t)Sx * Wy + Sy];
                if (fv == 0.0) continue;
                int p = (int)(Sx % Nx), q = (int)(Sy % Ny);
                const double* win = Hp + off + ((size_t)p * Ny + q) * ks * kt;
                for (int u = 0; u < ks; ++u) {
                    long X = Sx + u - cs;
                    if (X < 0 || X >= Wx) continue;
                    for (int v = 0; v < kt; ++v) {
                        long Y = Sy + v - ct;
                        if (Y < 0 || Y >= Wy) continue;
                        gz[(size_t)X * Wy + Y] += fv * win[(size_t)u * kt + v];
                    }
                }
            }
        off += depth_elems(Nx, Ny, ks, kt);
    }
    return 0;
}

/* g = H' f at selected voxels, one by one: pts holds npts triples (z, X, Y). */
int oracle_backproject_points(const double* Hp, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
                              const double* f, int Wx, int Wy, long npts, const int* pts,
                              double* out, int nthreads) {
    if (!Hp || !f || !pts || !out || !Ks || !Kt) return -1;
    set_threads(nthreads);
    size_t* off = (size_t*)malloc(sizeof(size_t) * (size_t)(Nz + 1));
    if (!off) return -2;
    off[0] = 0;
    for (int z = 0; z < Nz; ++z) off[z + 1] = off[z] + depth_elems(Nx, Ny, Ks[z], Kt[z]);
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < npts; ++i) {
        int z = pts[3 * i], X = pts[3 * i + 1], Y = pts[3 * i + 2];
        int ks = Ks[z], kt = Kt[z];
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        double acc = 0.0;
        for (int u = 0; u < ks; ++u) {
            long Sx = (long)X - u + cs;          /* pixels whose window holds X */
            if (Sx < 0 || Sx >= Wx) continue;
            for (int v = 0; v < kt; ++v) {
                long Sy = (long)Y - v + ct;
                if (Sy < 0 || Sy >= Wy) continue;
                int p = (int)(Sx % Nx), q = (int)(Sy % Ny);
                acc += f[(size_t)Sx * Wy + Sy]
                     * Hp[off[z] + (((size_t)p * Ny + q) * ks + u) * kt + v];
            }
        }
        out[i] = acc;
    }
    free(off);
    return 0;
}

/*
 * Gradient of L = sum_{X,z} (g(X,z) - g_ref(X,z))^2 with g = H' f, taken with
 * respect to the entries of H'.  With the residual r = 2 (g - g_ref) given as
 * [Nz][W_x][W_y]:  dL/dH'_z[p][q][u][v] = sum over pixels S with S mod N =
 * (p, q) of f(S) * r(S + (u - c_s, v - c_t), z), voxels outside the volume
 * contributing nothing.  Output in the H' layout, FP64.
 */
int oracle_grad_hp_f64(const double* f, const double* r, int Nx, int Ny, int Nz,
                       const int* Ks, const int* Kt, int Wx, int Wy, double* dHp, int nthreads) {
    if (!f || !r || !dHp || !Ks || !Kt) return -1;
    set_threads(nthreads);
    size_t* off = (size_t*)malloc(sizeof(size_t) * (size_t)(Nz + 1));
    if (!off) return -2;
    off[0] = 0;
    for (int z = 0; z < Nz; ++z) off[z + 1] = off[z] + depth_elems(Nx, Ny, Ks[z], Kt[z]);
    long nwork = (long)Nz * Nx * Ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (long w = 0; w < nwork; ++w) {
        int z = (int)(w / ((long)Nx * Ny));
        int p = (int)((w / Ny) % Nx), q = (int)(w % Ny);
        int ks = Ks[z], kt = Kt[z];
        int cs = (ks - 1) / 2, ct = (kt - 1) / 2;
        const double* rz = r + (size_t)z * Wx * Wy;
        for (int u = 0; u < ks; ++u)
            for (int v = 0; v < kt; ++v) {
                double acc = 0.0;
                for (long Sx = p; Sx < Wx; Sx += Nx) {
                    long X = Sx + u - cs;
                    if (X < 0 || X >= Wx) continue;
                    for (long Sy = q; Sy < Wy; Sy += Ny) {
                        long Y = Sy + v - ct;
                        if (Y < 0 || Y >= Wy) continue;
                        acc += f[(size_t)Sx * Wy + Sy] * rz[(size_t)X * Wy + Y];
                    }
                }
                dHp[off[z] + (((size_t)p * Ny + q) * ks + u) * kt + v] = acc;
            }
    }
    free(off);
    return 0;
}

/* oracle_grad_hp_f64 at selected entries, one by one: pts holds npts
 * 5-tuples (z, p, q, u, v); the residual r is [Nz][W_x][W_y]. */
int oracle_grad_hp_points(const double* f, const double* r, int Nx, int Ny, int Nz,
                          const int* Ks, const int* Kt, int Wx, int Wy, long npts,
                          const int* pts, double* out, int nthreads) {
    if (!f || !r || !pts || !out || !Ks || !Kt) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
    for (long i = 0; i < npts; ++i) {
        int z = pts[5 * i], p = pts[5 * i + 1], q = pts[5 * i + 2];
        int u = pts[5 * i + 3], v = pts[5 * i + 4];
        int cs = (Ks[z] - 1) / 2, ct = (Kt[z] - 1) / 2;
        const double* rz = r + (size_t)z * Wx * Wy;
        double acc = 0.0;
        for (long Sx = p; Sx < Wx; Sx += Nx) {
            long X = Sx + u - cs;
            if (X < 0 || X >= Wx) continue;
            for (long Sy = q; Sy < Wy; Sy += Ny) {
                long Y = Sy + v - ct;
                if (Y < 0 || Y >= Wy) continue;
                acc += f[(size_t)Sx * Wy + Sy] * rz[(size_t)X * Wy + Y];
            }
        }
        out[i] = acc;
    }
    return 0;
}
