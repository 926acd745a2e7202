/*
 * lfbp -- light-field backprojection arrays on one GPU (sm_103a).
 *
 * Builds the backprojection array H' from the shift-variant light-field PSF
 * array H as the pure re-arrangement derived in Eberhart, "Efficient
 * computation of backprojection arrays for 3D light field deconvolution"
 * (arXiv 2003.09133), Sec. 4, Eqs. (4)-(9): per depth, a flip of the pixel
 * axes of each cut-out combined with a cyclic exchange of the source
 * positions of the elementary cell.
 *
 * ARRAY LAYOUT (H, H' and their gradients alike).  One flat buffer per
 * array, depth-major and ragged in depth.  Depth z holds Nx*Ny*Ks[z]*Kt[z]
 * elements in row-major [a][b][s][t] order and starts at element
 * lfbp_plan_depth_offset(plan, z).  In H, (a, b) is the source position in
 * the elementary cell (the paper's x, y; Sec. 2.1, Sec. 4) and (s, t) the
 * pixel of the voxel-centred cut-out (the paper's s, t).  In H', (a, b) is
 * the pixel position inside the lenslet (the paper's x', y') and (s, t) the
 * voxel of the pixel-centred window (the paper's s', t').  The paper's x
 * pairs with s and y with t.
 *
 * THE MAP (default, LFBP_MAP_TRANSPOSE).  With c_s = (Ks-1)/2, c_t = (Kt-1)/2:
 *     H'[p][q][u][v] = H[(p+u-c_s) mod Nx][(q+v-c_t) mod Ny][Ks-1-u][Kt-1-v]
 * which is the transpose of the measurement operator of Eq. (1) stored
 * pixel-centred.  It is a permutation of each depth and its own inverse
 * (Sec. 4: processing H' gives back H).  Element values are moved as raw
 * bits (fp32 or fp16 storage); no arithmetic is done on them.
 *
 * LFBP_MAP_PAPER_WINDOW reproduces the loop ranges of Eqs. (4)-(9) literally
 * (m = 1..n_s): entries with p+u < h_x, p+u > Ks-1+h_x, q+v < h_y or
 * q+v > Kt-1+h_y (h = (N-1)/2) are written as zero bits instead.  In this
 * mode even cut-outs are taken as well (Eq. 8 then drops s = n_s and never
 * writes s' = n_s; see lfbp_plan_create2).
 *
 * Beside the map, the projectors that consume H' (Eqs. 1 and 2) and the
 * gradient with respect to H' run on fp32 plans (lfbp_backproject_volume and
 * the calls after it).
 *
 * CONVENTIONS.  All device pointers are owned by the caller and must stay
 * valid until the stream work completes.  Every call that takes a stream
 * enqueues asynchronous work on it (NULL = legacy default stream) and
 * returns without synchronising; an error inside a kernel is reported by
 * lfbp_sync_status.  Return values: LFBP_OK (0) or a negative LFBP_ERR_*;
 * lfbp_last_error() gives a message for the calling thread's last failure.
 * Plans are immutable after creation and may be shared between threads;
 * calls on the same plan from several threads are safe when they use
 * different output buffers.
 */
#ifndef LFBP_H
#define LFBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LFBP_F32 = 0, LFBP_F16 = 1 } lfbp_dtype;
typedef enum { LFBP_MAP_TRANSPOSE = 0, LFBP_MAP_PAPER_WINDOW = 1 } lfbp_mode;

#define LFBP_OK 0
#define LFBP_ERR_BAD_SHAPE (-1) /* even or non-positive N or K, too large a shape */
#define LFBP_ERR_NULL (-2)      /* a required pointer is NULL                     */
#define LFBP_ERR_ALIGN (-3)     /* a buffer does not start on a 16-byte boundary  */
#define LFBP_ERR_ALIAS (-4)     /* input and output buffers overlap               */
#define LFBP_ERR_DTYPE (-5)     /* unknown dtype or plans of mixed element size   */
#define LFBP_ERR_CUDA (-6)      /* a CUDA runtime call failed                     */
#define LFBP_ERR_TIMEOUT (-7)   /* a bounded in-kernel wait gave up               */
#define LFBP_ERR_NOMEM (-8)     /* host or device allocation failed               */
#define LFBP_ERR_INVALID (-9)   /* other invalid argument                         */

typedef struct lfbp_plan_s* lfbp_plan; /* opaque; owned by the library */

/*
 * Square elementary cell (Nx = Ny = Nnum, Ks = Kt = Kz[z]).  Nnum and every
 * Kz[z] must be odd and >= 1 (Sec. 4: n_x, n_y odd; odd n_s makes Eq. (8) a
 * flip, see lfbp_plan_create2).  Kz is copied.  Nz = 0 makes an empty plan:
 * the map calls (plain, batched, host, adjoint) return LFBP_OK for it at once,
 * with no CUDA call, and its buffers may be NULL.
 * On success *out receives a plan to be released with lfbp_plan_destroy.
 */
int lfbp_plan_create(lfbp_plan* out, int Nnum, int Nz, const int* Kz, lfbp_dtype dt,
                     lfbp_mode mode);

/*
 * General cell (Sec. 4: the x and y axes are mapped independently, so the
 * cell may be non-square, n_x != n_y, as for hexagonal MLAs): Nx x Ny source
 * positions, per-depth cut-outs of Ks[z] x Kt[z] pixels.  Nx, Ny odd, all
 * >= 1; Nx, Ny <= 1023 and Ks, Kt <= 16383.  Cut-outs must be odd for
 * LFBP_MAP_TRANSPOSE (LFBP_ERR_BAD_SHAPE otherwise).  In LFBP_MAP_PAPER_WINDOW
 * mode they may be even: Eq. (8) then drops one pixel row (s = n_s) and never
 * writes s' = n_s, and the map is the literal Eqs. (4)-(9) loop, a partial
 * injection.  A plan with an even cut-out is taken by lfbp_backproject_array
 * and lfbp_adjoint only (element by element, not tiled); the other entry
 * points reject it with LFBP_ERR_BAD_SHAPE.
 */
int lfbp_plan_create2(lfbp_plan* out, int Nx, int Ny, int Nz, const int* Ks, const int* Kt,
                      lfbp_dtype dt, lfbp_mode mode);

void lfbp_plan_destroy(lfbp_plan p);

/* Total elements of one array, sum_z Nx*Ny*Ks[z]*Kt[z]; 0 for a NULL plan. */
size_t lfbp_plan_elems(lfbp_plan p);
/* First element of depth z (0 <= z <= Nz; z = Nz gives lfbp_plan_elems). */
size_t lfbp_plan_depth_offset(lfbp_plan p, int z);
/* Bytes per element of the plan's dtype (4 or 2). */
int lfbp_plan_esize(lfbp_plan p);

/*
 * Split the plan's depths into nparts contiguous ranges of about equal
 * element counts (Sec. 4: the depths are independent), e.g. one per GPU:
 * part `part` (0 <= part < nparts) is depths [*z0, *z1), possibly empty.
 * Every boundary is the depth start nearest to its share; the ranges cover
 * 0..Nz without overlap.  Host only.  LFBP_ERR_NULL / LFBP_ERR_INVALID on bad
 * arguments.
 */
int lfbp_plan_partition(lfbp_plan p, int nparts, int part, int* z0, int* z1);

/*
 * H -> H' with one kernel launch per depth (Sec. 4: the z-planes are
 * independent).  dH, dHp: device buffers of lfbp_plan_elems(p) elements,
 * 16-byte aligned, not overlapping (in-place is rejected with
 * LFBP_ERR_ALIAS).  The plan's mode selects the full transpose or the
 * paper-window variant.
 */
int lfbp_backproject_array(lfbp_plan p, const void* dH, void* dHp, void* cuda_stream);

/*
 * H -> H' from host memory to host memory (Sec. 4: the z-planes are
 * independent, so the map streams through them in any order).
 * H_host, Hp_host: host buffers of lfbp_plan_elems(p) elements, not
 * overlapping.  Two paths:
 *  - default: host->device copies of fixed 64 MB byte ranges (aligned;
 *    LFBP_HOST_CHUNK_MB sets the size) on one library-owned helper stream,
 *    the map of each depth (one launch per depth, on cuda_stream) as soon as
 *    every range it overlaps has arrived, and device->host copies of
 *    each range once every depth overlapping it is mapped, on a second helper
 *    stream: both directions of the host link run at the same time.  The
 *    depths go in memory order; LFBP_HOST_ORDER=rotate (read at each call)
 *    takes them in a rotation that starts at the smallest depth.
 *    dH_work, dHp_work hold H and H' afterwards.  Page-locked (pinned) host
 *    memory is needed for the copies to overlap; pageable memory works.
 *  - LFBP_HOST_PATH=zerocopy in the environment (read at each call), with
 *    both buffers page-locked, mapped into the device's address space
 *    (cudaHostAlloc, cudaHostRegister, torch pinned tensors) and 16-byte
 *    aligned: one persistent launch reads H from host memory and writes H'
 *    to host memory itself (its loads are cp.async copies, not TMA).
 *    dH_work and dHp_work are validated but not touched.  Otherwise the
 *    default path runs.
 * dH_work, dHp_work: caller-owned device buffers of the plan's size, 16-byte
 * aligned, not overlapping.  All work is ordered after earlier work on
 * cuda_stream, and later work on cuda_stream waits for all of it (including
 * the last write to Hp_host); the call itself does not block.  The first
 * call on a device creates the helper streams (copy path) or the work list
 * (zero-copy path).
 */
int lfbp_backproject_array_host(lfbp_plan p, const void* H_host, void* Hp_host, void* dH_work,
                                void* dHp_work, void* cuda_stream);

/*
 * H -> H' for n arrays at once, as one CUDA graph launch over a ragged work
 * list of all depths of all arrays (mixed fp32 / fp16 plans allowed).  Sec. 4
 * maps each z-plane on its own (the index relations of Eqs. 4-9 never mix
 * depths), so the depths of several arrays form one list of independent
 * pieces of work, whatever their cell and cut-out sizes.  The launch takes
 * one of three forms (the autotuner's choice, lfbp_tune_batched; untuned:
 * one tile per CTA):
 *  - persistent CTAs that stream the tiles of the list through a ring of
 *    shared-memory stages (producer warps, consumer warps);
 *  - one grid over the whole list, one tile per CTA;
 *  - one grid per depth of every array, all in one graph with no dependencies
 *    between them.
 * The work list, launch shape and graph are built on the first call for a
 * given list of plans and reused while the same plans (by handle) come back;
 * pointers may change between calls.  The first call for a new list of plans
 * allocates device memory and must not be made during stream capture.
 * plans[i], dH[i], dHp[i] as for lfbp_backproject_array; no output may
 * overlap any input or other output.  With LFBP_LOADS=lsu in the environment
 * (read at each call) the persistent kernel's producers move the input
 * segments with 16-byte cp.async copies instead of TMA bulk copies, and the
 * persistent form is used; the result is the same.
 */
int lfbp_backproject_batched(int n, const lfbp_plan* plans, const void* const* dH,
                             void* const* dHp, void* cuda_stream);

/*
 * lfbp_backproject_batched without any device allocation (the paper has no
 * counterpart; this is a deployment aid).  Some callers cannot allocate
 * device memory on their own: a host application that hands out all device
 * memory from its own pool, or one that forbids cudaMalloc once its run has
 * started (allocation can synchronise the device and fail under memory
 * pressure at the worst moment).  This entry point keeps the persistent
 * kernel's work list in a fixed array of device memory that is part of the
 * library image: 262,144 tile descriptors (8 MiB), held on every GPU that
 * loads the library until the process exits.  A batch that needs more tiles
 * (even with tiles of at least 48 KiB) is rejected with LFBP_ERR_BAD_SHAPE
 * before any CUDA call.  The call never calls cudaMalloc or cudaFree and
 * builds no CUDA graph; it launches the kernel directly on cuda_stream.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and reads device attributes; make that first call
 * before any stream capture.  All calls share the one array, which keeps the
 * work list of the last call: when the plans differ from the previous call
 * on this device, the new list is copied in, in stream order, before the
 * launch (nothing in the array has to start at zero: the kernel reads only
 * the entries the current list occupies).  Calls whose work overlaps on the
 * GPU -- on different streams, or from threads that do not order their
 * streams -- race on the array and may map with the wrong list; keep such
 * calls on one stream or order them with events.  This holds for a call that
 * follows another on a different stream even when both name the same plans:
 * the later call finds the list already loaded and launches at once, so it
 * must be ordered after the earlier call (an event recorded after it) for the
 * earlier call's copy of the list to have landed.  A call that has to copy a
 * new list in returns LFBP_ERR_INVALID, without queuing work, while
 * cuda_stream is capturing: the copy reads host memory owned by the call.
 * Arguments, layout and results are those of lfbp_backproject_batched.
 */
int lfbp_backproject_batched_noalloc(int n, const lfbp_plan* plans, const void* const* dH,
                                     void* const* dHp, void* cuda_stream);

/*
 * Autotuner for lfbp_backproject_batched: times a small grid of launch shapes
 * (persistent CTAs: shared-memory bytes per tile in {12, 16, 24, 32, 40, 48,
 * 64} KiB x persistent CTAs per SM in {1, 2, 3, 4}; one tile per CTA, and a
 * graph of one grid per depth of every array: tile bytes in {24, 32, 40, 48,
 * 64} KiB; each with the pair consumer on or off) on
 * the given buffers with CUDA events (reps timed launches
 * each, after one warm-up) and keeps the fastest for later batched calls with
 * the same plans (by handle).  Writes H' into dHp as a side effect and
 * synchronises the stream.  If the environment variable LFBP_TUNE_CACHE names
 * a file, the choice is appended there, keyed by device name and array
 * shapes, and later processes take it from there without timing.  tuned
 * (may be NULL, else 5 ints) receives {tile bytes, CTAs per SM (0 unless
 * persistent), stages (0 = as many as fit), pair consumer (1 = on), form (0 =
 * persistent CTAs, 1 = one tile per CTA, 2 = per-depth grids in one graph)}.
 * Arguments otherwise as for lfbp_backproject_batched.  Without tuning,
 * LFBP_PAIRS=0 turns the pair consumer off and LFBP_FORM selects the form
 * (defaults: on, one tile per CTA with 64 KiB tiles; the result is the
 * same).
 */
int lfbp_tune_batched(int n, const lfbp_plan* plans, const void* const* dH, void* const* dHp,
                      void* cuda_stream, int reps, int* tuned);

/*
 * Adjoint of the plan's map, applied to a gradient with respect to H'
 * (dHp_grad) to give the gradient with respect to H (dH_grad).  For
 * LFBP_MAP_TRANSPOSE the map is its own inverse and its own adjoint
 * (Sec. 4, reversibility), so this is the same gather; for
 * LFBP_MAP_PAPER_WINDOW it gathers the unmasked entries and writes zeros
 * where the forward map dropped an entry.  Buffers as for
 * lfbp_backproject_array.
 */
int lfbp_adjoint(lfbp_plan p, const void* dHp_grad, void* dH_grad, void* cuda_stream);

/*
 * Scratch memory of the projector entry points below (backprojection,
 * forward projection, gradient, Richardson-Lucy update and normaliser): for
 * cut-outs of up to 9 cells per axis the kernels read their input tiles by
 * TMA tensor copies from a copy of the input laid out by phase (about the
 * size of the input image or volume).  That copy is allocated stream-ordered
 * on the call's stream from a memory pool the library creates per device (its
 * memory is kept for reuse, not returned to the system) and released on the
 * stream when the call's kernels are done.  When the pool cannot provide it,
 * the kernels read the input directly (same results, bit for bit).  The
 * environment variable LFBP_PROJ_TMA=0 selects the direct reads.
 */

/*
 * Backprojection of a sensor image through H' (the H' f inside the
 * Richardson-Lucy update, Eq. 2) on a finite Wx x Wy sensor whose voxel grid
 * coincides laterally with the pixel grid; the cell position of a point P is
 * P mod N and points outside the sensor contribute nothing:
 *   g[z][X][Y] = sum_{u,v} f[X-u+c_s][Y-v+c_t] * H'_z[(X-u+c_s) mod Nx][(Y-v+c_t) mod Ny][u][v]
 * dHp: H' in the plan's layout (LFBP_F32 plans only); df: [Wx][Wy] fp32;
 * dg: [Nz][Wx][Wy] fp32 output.  Sums run in fp32 in a fixed order
 * (deterministic).  Requires Kt <= 3072 (LFBP_ERR_BAD_SHAPE otherwise).
 */
int lfbp_backproject_volume(lfbp_plan p, const void* dHp, const float* df, int Wx, int Wy,
                            float* dg, void* cuda_stream);

/*
 * Forward projection f = H g (Eq. 1): every voxel adds its cut-out of H,
 * scaled by its value, onto the sensor (cut-out centred on the voxel):
 *   f[S] = sum_z sum_{s,t} g[z][S-s+c_s][.] * H_z[(S-s+c_s) mod Nx][..][s][t]
 * dH: H (LFBP_F32 plans only); dg: [Nz][Wx][Wy]; df: [Wx][Wy] output.
 * Depths are accumulated in order z = 0..Nz-1 (deterministic).
 */
int lfbp_forward_project(lfbp_plan p, const void* dH, const float* dg, int Wx, int Wy, float* df,
                         void* cuda_stream);

/*
 * Gradient of a loss L(g) with g = H' f (lfbp_backproject_volume) with respect
 * to the entries of H', given dL/dg ([Nz][Wx][Wy] fp32):
 *   dL/dH'_z[p][q][u][v] = sum over pixels S of cell (p, q) of f[S] * dL/dg_z[S + (u-c_s, v-c_t)]
 * df: [Wx][Wy]; dHp_grad: output in the plan's layout (fp32); it must not
 * overlap df or dgrad (LFBP_ERR_ALIAS).  Each output is a fixed-order fp32
 * sum (deterministic, no atomics).
 */
int lfbp_backproject_volume_grad(lfbp_plan p, const float* df, const float* dgrad, int Wx, int Wy,
                                 void* dHp_grad, void* cuda_stream);

/*
 * The same backprojection g = H' f as lfbp_backproject_volume, read straight
 * from H without building H' (Sec. 4's map substituted into the sum; for the
 * in-loop PSF updates of Sec. 3.1, where H' would otherwise be rebuilt every
 * iteration):
 *   g[z][X][Y] = sum_{s,t} f[X+s-c_s][Y+t-c_t] * H_z[X mod Nx][Y mod Ny][s][t]
 * dH: H in the plan's layout (LFBP_F32 plans); df: [Wx][Wy]; dg: [Nz][Wx][Wy]
 * output.  Equal to lfbp_backproject_volume on the mapped array up to the
 * order of the fp32 sums.  Requires Kt <= 3072.
 */
int lfbp_backproject_volume_from_h(lfbp_plan p, const void* dH, const float* df, int Wx, int Wy,
                                   float* dg, void* cuda_stream);

/*
 * One Richardson-Lucy update (Eq. 2):
 *   g_next = g / (H' 1) * [H' (f / (H g))]
 * The forward projection H g (as lfbp_forward_project) goes into dwork, is
 * replaced there by the quotient f / (H g) -- 0 where H g = 0 --, and the
 * quotient is backprojected with H' (as lfbp_backproject_volume); the
 * backprojection kernel's epilogue forms g / norm * sum (0 where norm = 0).
 * dH: H; dHp: H' = the plan's map of H (LFBP_F32 plan, transpose mode);
 * dnorm: H' 1 as [Nz][Wx][Wy] (lfbp_rl_normaliser); df: the measured image
 * [Wx][Wy]; dg: the estimate [Nz][Wx][Wy]; dg_next: the update, same shape --
 * it may be dg itself (every output reads only its own g), but must not
 * overlap any other buffer; dwork: Wx*Wy floats of caller-owned scratch.
 * fp32 sums in a fixed order (deterministic).  Requires Kt <= 3072.
 */
int lfbp_rl_step(lfbp_plan p, const void* dH, const void* dHp, const float* dnorm,
                 const float* df, int Wx, int Wy, const float* dg, float* dg_next, float* dwork,
                 void* cuda_stream);

/*
 * The update of lfbp_rl_step with H' never built: the backprojection reads H
 * directly (as lfbp_backproject_volume_from_h).  For estimates whose PSF
 * changes every iteration (Sec. 3.1: physics-updated or blind
 * deconvolution).  Arguments as for lfbp_rl_step without dHp.
 */
int lfbp_rl_step_fused(lfbp_plan p, const void* dH, const float* dnorm, const float* df, int Wx,
                       int Wy, const float* dg, float* dg_next, float* dwork, void* cuda_stream);

/*
 * The normaliser of Eq. 2, H' 1: the backprojection of a ones image on the
 * Wx x Wy sensor, into dnorm ([Nz][Wx][Wy]).  With dHp != NULL it uses H'
 * (lfbp_backproject_volume), else H directly (lfbp_backproject_volume_from_h).
 * dwork: Wx*Wy floats of scratch (filled with ones).
 */
int lfbp_rl_normaliser(lfbp_plan p, const void* dH, const void* dHp, int Wx, int Wy, float* dnorm,
                       float* dwork, void* cuda_stream);

/*
 * Synchronise the stream, then return and clear the library's device status
 * word for the current device: LFBP_OK, or LFBP_ERR_TIMEOUT when a bounded
 * in-kernel wait gave up (the output is then incomplete), or LFBP_ERR_CUDA
 * when the synchronisation itself failed.
 *
 * Tests of the error paths: the environment variable LFBP_FAULT (read at each
 * call) injects a failure -- "plan" (plan creation returns LFBP_ERR_NOMEM),
 * "alloc" (building a batch's work list returns LFBP_ERR_NOMEM), "graph" (its
 * graph instantiation returns LFBP_ERR_CUDA) or "stall" (persistent launches,
 * and the TMA copies of the projector kernels, are not issued, so their
 * bounded waits run out and this call returns LFBP_ERR_TIMEOUT some seconds
 * later).  Unset in normal use.
 */
int lfbp_sync_status(void* cuda_stream);

/* Message of the calling thread's last failed call ("" if none). */
const char* lfbp_last_error(void);

/* Library version string. */
const char* lfbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LFBP_H */
