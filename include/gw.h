/*
 * gw.h -- C ABI of the GB300 static-polarizability library (libgw.so).
 *
 * The library computes, on one GPU, the O(N^4) hot path of plane-wave GW as stated by Kim et
 * al., "Scalable GW software for quasiparticle properties using OpenAtom" (arXiv 1810.07772):
 *
 *   states psi_n(r), energies E_n
 *     -> pair densities f_vc(r) = conj(psi_v(r)) psi_c(r) sqrt(2/(E_c - E_v))      Eq. (fdef)
 *     -> P(r,r') = -sum_vc f_vc(r) conj(f_vc(r'))   (Hermitian rank-k update)     Eq. (Pstatic)
 *     -> P~(G,G') = sum_{r,r'} exp(-iG.r) P(r,r') exp(+iG'.r')  inside the sphere    Sec. 4.1
 *     -> eps = I - sqrt(V) P~ sqrt(V),  V(G) = 4 pi / (Omega |G|^2), V(0) = 0        Sec. 5.1
 *     -> eps^-1 (FP64)                                                             Sec. 5.1
 *
 * at q = 0 and one k-point, in Hartree atomic units.  Conventions shared by every call:
 *
 *   - Grid: n1 x n2 x n3 points, N_r = n1 n2 n3, index r = (j1 n2 + j2) n3 + j3 (C order).
 *     The cell is cubic with edge cell_L bohr (Omega = cell_L^3); position r = cell_L (j1/n1,
 *     j2/n2, j3/n3).
 *   - G-vectors: G = 2 pi m / cell_L for integers m in FFT range ([-n/2, n - n/2) per axis).
 *     The eps basis is every m with |m|^2 <= gcut, ordered by (|m|^2, m1, m2, m3) ascending,
 *     so G = 0 is entry 0.
 *   - Complex numbers are interleaved (re, im): complex64 = 2 x float, complex128 = 2 x double.
 *     Matrices are row-major and dense (leading dimension = number of columns).
 *
 * Calls are asynchronous on the context's CUDA stream unless stated; device pointers must be
 * valid on the context's device.  Every call returns a gw_status and never aborts, throws or
 * traps.  Errors raised inside kernels (a wait that ran out, a non-positive Cholesky pivot) are
 * recorded in a device status word and reported by the next synchronising call (gw_eps_inv,
 * gw_sync).  One context must not be used by two host threads at once.
 */
#ifndef GW_H
#define GW_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GW_API __attribute__((visibility("default")))
#else
#define GW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gw_status {
    GW_OK = 0,
    GW_E_INVALID = 1,     /* bad argument: size, pointer, NaN/Inf, E_v >= E_c, ...           */
    GW_E_NOMEM = 2,       /* device allocation failed                                        */
    GW_E_CUDA = 3,        /* a CUDA runtime call failed (message in gw_last_error)           */
    GW_E_NOT_READY = 4,   /* call-order violation: e.g. gw_build_P before gw_load_states      */
    GW_E_NUMERIC = 5,     /* eps is not Hermitian positive definite (Cholesky pivot <= 0)    */
    GW_E_TIMEOUT = 6,     /* a bounded device-side wait ran out; the kernel returned early   */
    GW_E_UNSUPPORTED = 7  /* valid request this build does not provide                       */
} gw_status;

/* Arithmetic used for the Hermitian rank-k update P = -F^T conj(F).                         */
typedef enum gw_precision {
    GW_PREC_TF32X3 = 0,    /* DIAGNOSTIC, not a plain-FP32 mode: tcgen05 kind::tf32, every FP32 */
                           /* operand split x = hi + lo, both rounded to TF32, hi*hi + hi*lo +   */
                           /* lo*hi, one TMEM accumulation over all k.  The truncating FP32 sum  */
                           /* of that one accumulation limits accuracy to ~1e-8 * k/8 (2.2e-4 on */
                           /* P~ at k = 15360), so it misses a 1e-6 target; GW_PREC_FP16X3 is the */
                           /* mode that meets it.  Kept to measure what window promotion buys.    */
    GW_PREC_BF16X3 = 1,    /* tcgen05 kind::f16 (BF16); same split and promotion as FP16X3       */
    GW_PREC_TF32X1 = 2,    /* tcgen05 kind::tf32, one product (diagnostic, ~1e-4 relative)      */
    GW_PREC_FP32_SIMT = 3, /* plain FP32 FMA on the CUDA cores (the same-GPU FP32 comparison)   */
    GW_PREC_FP16X3 = 4     /* tcgen05 kind::f16 (FP16) with one global power-of-two scale; the   */
                           /* three-product split, short TMEM windows promoted to FP32 registers */
} gw_precision;

typedef enum gw_inv_method {
    GW_INV_CHOLESKY = 0,   /* FP64 blocked Cholesky eps = L L^H, then eps^-1 = L^-H L^-1        */
    GW_INV_NEWTON = 1,     /* FP64 Newton iteration X <- X (2I - eps X) of Sec. 5.1, from        */
                           /* X0 = eps^H / max_i sum_j |(eps eps^H)_ij|, until max |dX| < 1e-11  */
    GW_INV_NEWTON_TC = 2   /* the Newton iteration of Sec. 5.1 on the 16-bit tensor cores, for a  */
                           /* Hermitian positive definite eps: FP16X3 steps from the Jacobi-scaled */
                           /* X0 = 2/(1+u) diag(eps)^-1 (u = max row sum of the scaled |eps|) to  */
                           /* max |I - eps X| < 3e-5, then two                                     */
                           /* refinements R = I - eps X, X <- X + X R with R exact to FP64 from   */
                           /* integer slices (see gw_zgemm_tc); GW_E_NUMERIC if the residual      */
                           /* before the last refinement exceeds 1e-8.  gw_eps_inv replays it     */
                           /* from a CUDA graph with 8 FP16X3 steps queued; an eps that needs    */
                           /* more is finished by the eager form (up to 16, host-checked)         */
} gw_inv_method;

typedef enum gw_dtype { GW_C64 = 0, GW_C128 = 1 } gw_dtype;

typedef struct gw_ctx gw_ctx;

/* Static string for a status code (never NULL). */
GW_API const char *gw_status_str(int status);

/* ABI version of this header: 1. */
GW_API int gw_version(void);

/*
 * Create a context on CUDA device `device`, enqueuing on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The context owns every internal device buffer; they are freed by
 * gw_destroy.  *out is set to NULL on failure.
 */
GW_API gw_status gw_create(gw_ctx **out, int device, void *stream);
GW_API gw_status gw_destroy(gw_ctx *ctx);
GW_API gw_status gw_set_stream(gw_ctx *ctx, void *stream);

/* Copy the last error message of this context into buf (NUL-terminated, at most n bytes). */
GW_API gw_status gw_last_error(const gw_ctx *ctx, char *buf, size_t n);

/*
 * Load the states and energies (Sec. 3 item 1: the DFT input).  Eq. (fdef) at q = 0.
 *   psi          [nv + nc][N_r] complex, occupied states first, r contiguous.  Stored on the
 *                device as complex64 (complex128 input is rounded).  psi_on_device != 0 means
 *                a device pointer, else a host pointer (copied synchronously to the stream).
 *   energies_eV  host array [nv + nc] in eV (divided by 27.211386245988 to Hartree); the
 *                weights 2 / (E_c - E_v) are formed in FP64 on the device.
 * Requires nv, nc >= 1, n1, n2, n3 in [2, 64], nv + nc <= N_r, cell_L > 0, finite energies and
 * max(E_v) < min(E_c); otherwise GW_E_INVALID.  The buffers are borrowed for the call only.
 * Invalidates any P, P~ or eps of an earlier load.
 */
GW_API gw_status gw_load_states(gw_ctx *ctx, int n1, int n2, int n3, double cell_L, int nv, int nc,
                         const void *psi, int psi_dtype, int psi_on_device,
                         const double *energies_eV);

/*
 * Form the pair densities and the Hermitian rank-k update (Eq. fdef and the outer product of
 * Sec. 4.1; Eq. Pstatic):  P(r,r') = -sum_{v,c} f_vc(r) conj(f_vc(r')).
 *   precision  a gw_precision.
 *   P_out      NULL, or a device buffer of N_r x N_r complex64 that receives a copy of P.
 * P itself stays in the context (full Hermitian matrix, both triangles written, real diagonal)
 * and can be read with gw_get_buffer(GW_BUF_P).  Requires gw_load_states.
 */
GW_API gw_status gw_build_P(gw_ctx *ctx, int precision, void *P_out);

/*
 * The row and column transforms of Sec. 4.1, restricted to the sphere |m|^2 <= gcut:
 *   P^(G, r') = sum_r exp(-i G.r) P(r, r'),  P~(G, G') = sum_r' P^(G, r') exp(+i G'.r').
 *   ng_out    host int, receives N_g.
 *   gvec_out  NULL or host int array [N_g][3] receiving the integer vectors m in basis order
 *             (up to max_ng entries are written when gvec_out != NULL; GW_E_INVALID if
 *             N_g > max_ng).
 *   PG_out    NULL or a device buffer of N_g x N_g complex64 receiving P~.
 * Requires gw_build_P.  gcut must keep the sphere inside the grid: 4 gcut < min(n_i)^2.
 */
GW_API gw_status gw_P_to_G(gw_ctx *ctx, int gcut, int *ng_out, int *gvec_out, int max_ng, void *PG_out);

/*
 * P~ without P(r,r'): the g-space route of Sec. 4.1 (Eq. gpsaceP), written with the pair
 * densities of Eq. (fdef):
 *   M_k(G) = sum_r exp(-i G.r) f_k(r)       (sphere transform of each pair density),
 *   P~(G, G') = -sum_k M_k(G) conj(M_k(G'))  (Hermitian rank-k update of N_g x N_g).
 * It equals gw_build_P followed by gw_P_to_G in exact arithmetic, and needs about
 * N_g^2 / N_r^2 of its rank-k work (plus k sphere transforms).
 *   precision  GW_PREC_FP16X3 or GW_PREC_BF16X3: the update runs on the 16-bit tensor-core kernel
 *              with the operand scaled by a power of two from max |M|.
 *   gcut, ng_out, gvec_out, max_ng, PG_out  as gw_P_to_G.
 * Requires gw_load_states; afterwards gw_eps_inv may be called, while P (GW_BUF_P) is not
 * available until gw_build_P.  Device memory: k N_r + k N_g complex64 and the 16-bit planes.
 * Timing slots (gw_get_times): [0] pair densities, [2] their sphere transforms, [3] the N_g
 * update.
 */
GW_API gw_status gw_build_PG(gw_ctx *ctx, int precision, int gcut, int *ng_out, int *gvec_out, int max_ng,
                             void *PG_out);

/*
 * eps_GG' = delta_GG' - sqrt(V(G)) P~_GG' sqrt(V(G')) and its inverse, both complex128 and
 * formed in FP64 (Sec. 5.1).  eps_out / epsinv_out: NULL, or N_g x N_g complex128 buffers on
 * the device or the host (host buffers are filled before the call returns).  This call
 * synchronises the stream and returns any device-side status (GW_E_NUMERIC if a Cholesky
 * pivot is <= 0, GW_E_TIMEOUT if a kernel wait ran out).  Requires gw_P_to_G.
 * GW_INV_NEWTON_TC is captured into a CUDA graph on the first call for an order N_g (on a private
 * stream of the context; the capture synchronises the context's stream once) and replayed on the
 * context's stream afterwards.  Because of the synchronisation the call cannot be made while the
 * context's stream is being captured: it then returns GW_E_INVALID before queuing anything.
 */
GW_API gw_status gw_eps_inv(gw_ctx *ctx, int method, void *eps_out, void *epsinv_out);

/* Synchronise the context stream and return the device-side status word (then clear it). */
GW_API gw_status gw_sync(gw_ctx *ctx);

/* Internal buffers, exposed read-only for inspection and tests.                               */
typedef enum gw_buffer {
    GW_BUF_P = 0,        /* N_r x N_r complex64, P(r, r')                                      */
    GW_BUF_F = 1,        /* pair-density operand planes, layout described below                */
    GW_BUF_PG = 2,       /* N_g x N_g complex64, P~                                             */
    GW_BUF_EPS = 3,      /* N_g x N_g complex128, eps                                           */
    GW_BUF_EPSINV = 4,   /* N_g x N_g complex128, eps^-1                                        */
    GW_BUF_WEIGHTS = 5,  /* [nv][nc] float, sqrt(2 / (E_c - E_v)) in Hartree^-1/2              */
    GW_BUF_PSIT = 6      /* [N_r][nv + nc] complex64, the loaded states transposed (r major)     */
} gw_buffer;

/*
 * Return the device pointer and byte size of an internal buffer (GW_E_NOT_READY if it has not
 * been produced yet).  Pointers stay valid until the next gw_load_states or gw_destroy.
 *
 * GW_BUF_F layout (precisions TF32X3 / TF32X1): float planes, k = v * nc + c padded with zeros
 * to a multiple of 8 (kpad), rows padded with zeros to a multiple of 256 (nr_pad).  For chunk
 * kc = k / 8 and plane p (0 = Re hi, 1 = Re lo, 2 = Im hi, 3 = Im lo; TF32X1 keeps only
 * p = 0 and 2, stored as planes 0 and 1), the element (r, k) sits at float offset
 *   ((kc * nplanes + p) * nr_pad + (r / 8) * 8) * 8 + ((k % 8) / 4) * 32 + (r % 8) * 4 + k % 4.
 * For GW_PREC_FP32_SIMT it is [kpad][nr_pad] complex64 (f itself, r contiguous).
 * For GW_PREC_FP16X3 / GW_PREC_BF16X3 it is 16-bit planes (FP16 or BF16 bit patterns; FP16
 * values carry the factor 2^e of the scale), k padded to a multiple of 16, stored block by block:
 * for kc = k / 16 and the 128-row block r / 128 the block's npl planes lie side by side, and the
 * element (r, k) of plane slot p sits at 16-bit offset
 *   ((kc * (nr_pad / 128) + r / 128) * npl + p) * 2048 + ((r % 128) / 8) * 128
 *       + ((k % 16) / 8) * 64 + (r % 8) * 8 + k % 8.
 * GW_HERK_SINGLE: npl = 4, slots Im hi, Re hi, Im lo, Re lo.  GW_HERK_PAIR: npl = 6, slots Im hi,
 * Im lo, Re hi, Re lo, -Im hi, -Im lo (the last two the first two with the sign bit flipped).
 */
GW_API gw_status gw_get_buffer(gw_ctx *ctx, int which, void **ptr, size_t *bytes);

/* Sizes of the loaded problem: dims[0..7] = n1, n2, n3, N_r, nv, nc, N_g (0 before gw_P_to_G),
 * nr_pad. */
GW_API gw_status gw_get_dims(gw_ctx *ctx, int *dims8);

/*
 * Per-kernel device times (ms) of the most recent gw_build_P / gw_P_to_G / gw_eps_inv, taken
 * with CUDA events on the context stream when timing is enabled (gw_set_timing(ctx, 1)); the
 * events never block the calls, they are read at the next synchronisation.  times[0] = pair
 * densities, [1] = rank-k update, [2] = row transform, [3] = conjugate transpose, column
 * transform and Hermitian part, [4] = eps build, [5] = eps inverse.  Synchronises the stream.
 * gw_reset_times clears the running means reported by gw_get_stats.
 */
GW_API gw_status gw_set_timing(gw_ctx *ctx, int enable);
GW_API gw_status gw_get_times(gw_ctx *ctx, float *times6);
GW_API gw_status gw_reset_times(gw_ctx *ctx);

/*
 * Counters (synchronises the stream): stats8[0] = kernels this library has launched in this
 * process, [1] = Newton iterations of the last GW_INV_NEWTON inverse (FP16X3 steps for
 * GW_INV_NEWTON_TC and gw_zinv_tc), [2] = mean rank-k update
 * time in ms over the timed calls since gw_reset_times, [3] = number of those calls, [4] = the
 * FP16 scale exponent e of the last 16-bit build, [5] = rank-k update tiles (CTA pairs for
 * GW_HERK_PAIR), [6] and [7] = the window and flush lengths of the 16-bit update.
 */
GW_API gw_status gw_get_stats(gw_ctx *ctx, double *stats8);

/*
 * Batch of independent systems (several q-points or supercells of uneven size), each held by its
 * own context with its states loaded.  A batch pass computes, for every instance, the same results
 * as gw_build_P (16-bit precisions) + gw_P_to_G + gw_eps_inv(GW_INV_CHOLESKY):
 *   - pair densities per instance;
 *   - ONE persistent launch of the rank-k update over the tiles of every instance (one CTA per SM
 *     walks a static tile list ordered by decreasing k), bit-identical to the per-instance kernel
 *     for the same window settings;
 *   - per-instance transforms, eps and FP64 inverse.
 * Results are read from each context (gw_get_buffer GW_BUF_PG / GW_BUF_EPSINV, or gw_eps_inv-style
 * buffers via gw_get_buffer).  All contexts must share one device and one stream.
 *
 * gw_batch_create   ctxs[n] loaded contexts, gcuts[n] their sphere cuts, precision GW_PREC_FP16X3
 *                   or GW_PREC_BF16X3 (else GW_E_UNSUPPORTED).  Allocates every buffer the pass
 *                   needs, builds the sphere plans and the tile table.  The contexts must outlive
 *                   the batch and must not be reloaded while it is in use.
 * gw_batch_run      one pass.  use_graph != 0: the first call runs eagerly, the second captures the
 *                   whole pass into a CUDA graph, later calls replay it (recaptured after
 *                   gw_batch_set_window).  Synchronises the stream and returns the first error
 *                   of any instance (message: gw_batch_last_error).
 * gw_batch_autotune picks the window / flush lengths of the rank-k update by timing the candidates
 *                   whose measured FP16-split error x 1.25 is within target_error (e.g. 1e-6); the
 *                   choice is appended to cache_path (JSON lines keyed by the instance shapes and the
 *                   target; NULL = no cache) and reused from it when the same batch is tuned again
 *                   for the same target.
 * gw_batch_stats    stats4[0] = last pass's rank-k update time in ms, [1] = window, [2] = flush,
 *                   [3] = number of tiles.
 */
typedef struct gw_batch gw_batch;
GW_API gw_status gw_batch_create(gw_batch **out, gw_ctx *const *ctxs, int n, const int *gcuts, int precision);
GW_API gw_status gw_batch_destroy(gw_batch *batch);
GW_API gw_status gw_batch_run(gw_batch *batch, int use_graph);
GW_API gw_status gw_batch_set_window(gw_batch *batch, int window_chunks, int flush_windows);
GW_API gw_status gw_batch_autotune(gw_batch *batch, const char *cache_path, double target_error);
GW_API gw_status gw_batch_stats(gw_batch *batch, double *stats4);
/* eps^-1 of every instance: GW_INV_NEWTON_TC (the default; its steps are all queued and the
 * unneeded ones return at once on the device, so the pass stays one CUDA graph) or
 * GW_INV_CHOLESKY.  Re-prepares the batch's buffers; GW_E_INVALID for another method. */
GW_API gw_status gw_batch_set_inverse(gw_batch *batch, int method);
GW_API gw_status gw_batch_last_error(const gw_batch *batch, char *buf, size_t n);

/*
 * Allocation-free inverse of a Hermitian positive-definite complex128 matrix, by the same FP64
 * blocked Cholesky that gw_eps_inv uses.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- applications whose device memory belongs to another
 * allocator (a framework's caching pool or an arena sized at start-up, where a raw cudaMalloc
 * fragments the pool or fails once it has claimed everything), and loops that must not pay
 * cudaFree's device-wide synchronisation.
 *   eps     device pointer, n x n complex128, row-major (only its lower triangle is read)
 *   n       1 <= n <= 512; larger orders return GW_E_INVALID
 *   epsinv  device pointer, n x n complex128, receives eps^-1 (both triangles written)
 *   stream  cudaStream_t to enqueue on (NULL = legacy default stream)
 * The call reads its status word back to the host and synchronises `stream` before it returns, so
 * the calling thread blocks until the inverse is done; it returns GW_E_NUMERIC if a Cholesky pivot
 * was <= 0.  Both pointers must be device memory of the calling thread's current device, else
 * GW_E_INVALID.  No context is needed and no device memory is allocated: the workspace is one
 * static device array of 12.9 MB, which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address; make that first call
 * before any stream capture.  All calls share the array and it keeps the last call's contents (the
 * call clears what must start at zero), so calls that overlap on the GPU (other threads, other
 * streams) race: serialise them.
 */
GW_API gw_status gw_eps_inv_noalloc(const void *eps, int n, void *epsinv, void *stream);

/*
 * States given as plane-wave coefficients (the DFT input of Sec. 4.1, u_nk(x) =
 * sum_g u~_nk(g) e^{i g.x} / sqrt(Omega)).  The library transforms them to the grid,
 *     psi_n(r_j) = N_r^(-1/2) sum_p coef[n][p] exp(+2 pi i (m1 j1/n1 + m2 j2/n2 + m3 j3/n3)),
 * (m = gvec_psi[p], taken modulo the grid; unit-norm coefficient vectors give unit-norm states),
 * in FP32 on the GPU, then loads them exactly as gw_load_states does.
 *   npw        number of plane waves, 1 <= npw <= N_r
 *   gvec_psi   host int [npw][3] Miller indices; two that coincide modulo the grid are
 *              GW_E_INVALID (they would alias)
 *   coef       [nv + nc][npw] complex (GW_C64 or GW_C128), host or device (coef_on_device)
 *   other arguments as gw_load_states (the grid also bounds the transform: n1, n2, n3 <= 64).
 * The call synchronises the stream.
 */
GW_API gw_status gw_load_states_g(gw_ctx *ctx, int n1, int n2, int n3, double cell_L, int nv, int nc, int npw,
                                  const int *gvec_psi, const void *coef, int coef_dtype, int coef_on_device,
                                  const double *energies_eV);

/*
 * Sums over k-points (Sec. 4.1: P^q = (1/N_k) sum_k of the one-k-point sums).  The P~ that the
 * next gw_P_to_G or gw_build_PG forms is multiplied by `weight` (e.g. 1/N_k) and, with accumulate
 * = 1, added to the P~ the previous of those calls left (the running sum); gw_eps_inv then uses the
 * sum.  With accumulate = 1 the sphere must be the one of that previous P~ (GW_E_INVALID
 * otherwise; GW_E_NOT_READY if there is none).  For each k-point the caller loads the states
 * (u_{v,k+q} occupied, u_{c,k} unoccupied) and sets q as for one k-point.  The setting persists
 * until changed; the default is weight 1, accumulate 0.  Non-finite weights are GW_E_INVALID.
 */
GW_API gw_status gw_set_kweight(gw_ctx *ctx, double weight, int accumulate);

/*
 * The plasmon-pole model of Sec. 5.2 (von der Linden-Horsch form) from the last gw_eps_inv:
 *   S = sqrt(V) (eps^-1 - I) sqrt(V) (Hermitian, negative semidefinite since eps >= I), its nmodes
 *   most negative eigenvalues sigma_a (ascending) and orthonormal eigenvectors A[:, a]
 *   (Eq. eigdecomp), by block subspace iteration with Rayleigh-Ritz in FP64 until every
 *   || S a - sigma_a a || <= tol |sigma_0|;
 *   the mode frequencies of the Johnson sum rule (Eq. ppfreq),
 *     omega_a^2 = -(1/sigma_a) sum_{g,g'} conj(A_ga) V(q+g) V(q+g') ((q+g).(q+g')) rho(g - g') A_g'a,
 *   Hartree^2, with rho(G) = sum_r e^{-iG.r} 2 sum_v |psi_v(r)|^2 the density of the loaded
 *   occupied states (rho(0) = 2 N_v electrons per cell); g - g' is taken modulo the grid.  The
 *   minus sign makes omega^2 > 0 (sigma < 0, the density form is positive semidefinite).
 *   nmodes 1..16 (and <= N_g); tol > 0.  Outputs may be NULL: sigma, omega2, resid [nmodes] on the
 *   host, A_out [N_g][nmodes] complex128 (host or device).  Needs gw_eps_inv and the states it was
 *   built from; GW_E_NUMERIC if the iteration does not converge (400 iterations).
 */
GW_API gw_status gw_pp_modes(gw_ctx *ctx, int nmodes, double tol, double *sigma, double *omega2, double *resid,
                             void *A_out);

/*
 * S(omega) = sum_{a < nuse} A_a sigma_a omega_a^2 / (omega_a^2 - omega^2) A_a^H (Eq. ppform) from
 * the last gw_pp_modes (nuse <= its nmodes); omega in Hartree; S_out N_g x N_g complex128, host or
 * device.  With every mode at omega = 0 it is S itself.
 */
GW_API gw_status gw_pp_eval(gw_ctx *ctx, double omega, int nuse, void *S_out);

/*
 * Complex GEMM C = A B from FP64 operands on the 16-bit tensor cores (the products of the
 * GW_INV_NEWTON_TC inverse).  Each operand is scaled by one power of two 2^e (max |Re|, |Im| <
 * 2^e) and sliced:
 *   mode 0  FP16X3: y = x 2^(14 - e), hi = rn16(y), lo = rn16(y - hi); hi*hi + hi*lo + lo*hi
 *           accumulated in FP32 (about 1e-6 relative, normwise);
 *   mode 1  integer slices (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012): x 2^-e =
 *           sum_t a_t 2^(-6(t+1)) + r with a_0 in [-64, 64], a_t in [-32, 31], nine slices; every
 *           slice product and every partial sum of a work slot is an integer below 2^24, so the
 *           tensor cores sum exactly and the result has FP64 accuracy (error about
 *           K 2^-54 max|A| max|B| per entry; integer-valued inputs below 2^6 give exact results).
 *   A, B, C   device pointers, complex128, row-major: A is M x K with row stride lda, B is K x N
 *             with row stride ldb, C is M x N with row stride N (written, not read)
 *   1 <= M, N, K <= 16384.  Uses the context's stream and workspace and synchronises it.
 */
GW_API gw_status gw_zgemm_tc(gw_ctx *ctx, int mode, int M, int N, int K, const void *A, int lda, const void *B,
                             int ldb, void *C);

/*
 * Inverse of a Hermitian positive definite complex128 matrix by the GW_INV_NEWTON_TC iteration.
 *   A  device pointer, n x n complex128, row-major; X receives A^-1 (device, n x n)
 *   1 <= n <= 16384.  Returns GW_E_NUMERIC when the iteration does not reach the FP64 refinement
 * (A not positive definite, or too ill-conditioned for 16 FP16X3 steps).  The number of FP16X3
 * steps taken is reported by gw_get_stats (stats8[1]).
 */
GW_API gw_status gw_zinv_tc(gw_ctx *ctx, int n, const void *A, void *X);

/* Report of the last GW_INV_NEWTON_TC inverse or gw_zinv_tc call on this context (-1 before
 * any): out4[0] = FP16X3 Newton steps of phase 1 (16 = the limit, reached without converging),
 * [1] = max |I - A X| after phase 1 (measured to FP64 accuracy), [2] = the last measured residual
 * (the one before the last correction), [3] = refinements that ran (1..3). */
GW_API gw_status gw_newton_tc_report(gw_ctx *ctx, double *out4);

/*
 * Window length of the 16-bit rank-k update: the tensor core accumulates `window_chunks` chunks
 * of 16 k (1..64, default 3) in TMEM before they are added into FP32 registers, and every
 * `flush_windows` windows (1..4096, default 256) the registers are added into P.  Shorter windows
 * and flushes mean smaller accumulation error.
 */
GW_API gw_status gw_set_herk_window(gw_ctx *ctx, int window_chunks, int flush_windows);

/*
 * Kernel of the 16-bit rank-k update of gw_build_P (Eq. Pstatic; the outer product of Sec. 4.1).
 * Both compute the same numbers (the same products and accumulation order per element):
 *   GW_HERK_PAIR    clusters of two CTAs share each tensor-core operation (2-SM MMAs,
 *                   M = 256): each CTA holds 128 rows of A and half of B, 256 x 128 complex tiles;
 *                   the operand holds six 16-bit planes per k chunk (the Im planes also negated)
 *   GW_HERK_SINGLE  (default) one CTA per 128 x 128 complex tile, four planes per k chunk
 * Takes effect at the next gw_build_P; GW_E_INVALID for another value.
 */
enum { GW_HERK_SINGLE = 0, GW_HERK_PAIR = 1 };
GW_API gw_status gw_set_herk_kernel(gw_ctx *ctx, int kind);

/*
 * Kernel of the sphere transforms (the two FFT phases of Sec. 4.1, pruned to the eps sphere) in
 * gw_P_to_G, gw_build_PG and the batch:
 *   GW_TRANSFORM_TWO_KERNEL (default) planes transformed over j3 and j2 into a workspace, then j1 per
 *                           row; where n2 = n3 is 12, 16, 18, 20, 24 or 27 and the sphere is
 *                           centred (q = 0) with max |m3| <= 7, the j3 and j2 sums take their
 *                           twiddles as compile-time constants, else from tables in shared memory
 *   GW_TRANSFORM_TABLES     the two-kernel form with twiddle tables everywhere (the form of the
 *                           other grids), kept for comparison
 *   GW_TRANSFORM_FUSED      one kernel per pass: each row is streamed plane by plane into shared
 *                           memory by bulk copies and transformed axis by axis (j1, j2, j3) there,
 *                           reading P from HBM exactly once; used where N_r and n2 n3 are even and
 *                           max |m| <= 8, else the two-kernel form.  Measured slower at 24^3
 *                           (0.96 against 0.83 ms for the row pass; equal on the g-space route)
 * All give the same sums up to FP32 rounding.  GW_E_INVALID for another value.
 */
enum { GW_TRANSFORM_TWO_KERNEL = 0, GW_TRANSFORM_FUSED = 1, GW_TRANSFORM_TABLES = 2 };
GW_API gw_status gw_set_transform_kernel(gw_ctx *ctx, int kind);

/*
 * Error target of the 16-bit rank-k update, as the relative Frobenius error of P~ against FP64
 * (0 = use the window of gw_set_herk_window, the default).  Each gw_build_P / gw_build_PG then
 * takes the longest window of 16, 8, 6, 5, 4, 3, 2, 1 chunks whose predicted error x 1.25 meets
 * the target at the call's precision; the predictions are errors measured at 24^3 (FP16X3:
 * 2.9e-7 at 1 chunk, 6.5e-7 at 3, 3.3e-6 at 16; BF16X3 4e-6 above those).  The flush length
 * stays that of gw_set_herk_window.  GW_E_INVALID for a negative or non-finite target,
 * GW_E_UNSUPPORTED when no window meets it (below 3.6e-7); a build whose precision cannot meet
 * it fails with GW_E_UNSUPPORTED.  gw_set_herk_window clears the target.  The window used is
 * reported by gw_get_stats (stats8[6]).
 */
GW_API gw_status gw_set_error_target(gw_ctx *ctx, double target);

/*
 * Wave vector q of eps^q (Sec. 4.1 and 5.1), in units of 2 pi / cell_L per axis (default 0).
 * eps^q_GG' = delta_GG' - sqrt(V(q+G)) P~^q_GG' sqrt(V(q+G')), V(q+G) = 4 pi / (Omega |q+G|^2); only
 * where q + G = 0 (the head at q = 0) is V set to 0.  For q != 0 the states passed to
 * gw_load_states are periodic parts: the occupied rows u_{v,k+q} with energies E_{v,k+q}, the
 * unoccupied rows u_{c,k} with E_{c,k}; the pair densities and transforms are the same as at q = 0
 * (they need no orthogonality between the two sets).  V is recomputed at once for the current
 * sphere (the call synchronises the context's stream), so the next gw_eps_inv uses it; P~ depends
 * on q only through the states the caller loads.
 */
GW_API gw_status gw_set_q(gw_ctx *ctx, const double *q);

/* Upper bound, in milliseconds, of any single device-side wait (default 2000).  A wait that
 * runs out makes its kernel record GW_E_TIMEOUT and return early. */
GW_API gw_status gw_set_wait_limit(gw_ctx *ctx, double ms);

/* ------------------------------------------------------------------------------------------
 * Learned truncation correction.
 *
 * In practice the sum over unoccupied states c in Eq. (Pstatic) is cut at N_c = nc_keep, and
 * Sec. 2 counts this band truncation among the method's costs.  The paper gives no correction;
 * this library adds a learned one.  A multilayer perceptron
 *     h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3), y = W4 h3 + b4
 * (n_in -> hidden -> hidden -> hidden -> 2) maps features x of one upper-triangle entry
 * (g, h), g <= h, of the truncated P~ to y ~ s (P~_all - P~_keep)(g, h) as (Re, Im).
 *
 * Weights are used in FP16 (rounded from an FP32 master copy), biases and accumulation in FP32.
 *
 * Upper-triangle entries are stored row-major: entry (g, h) is row t = g ng - g (g - 1)/2 + (h - g),
 * and there are ng (ng + 1)/2 rows.
 *
 * Scale s = 1 / mean_{g >= 1} |Re P~_keep(g, g)|.  It makes features and targets O(1) for any
 * system.
 *
 * Features (float32, 12 per row):
 *   [ |m_g|^2/gcut, |m_h|^2/gcut, |m_g - m_h|^2/(4 gcut), s Re P~(g,h), s Im P~(g,h), s Re P~(g,g),
 *     s Re P~(h,h), [g == h], ratio, [g == 0 or h == 0], s Re dP~(g,h), s Im dP~(g,h) ]
 * Here m are the integer G-vectors, ratio is the per-system scalar from gw_corr_weight_ratio and
 * dP~ the closure estimate of the omitted part (gw_corr_closure; zero when not given).  With a
 * closure estimate the network learns what it leaves: targets s (P~_all - P~_keep - dP~), and the
 * learned form is P~_keep + dP~ + y / s.
 *
 * Parameters are one flat float32 vector [W1, b1, W2, b2, W3, b3, W4, b4], each W_l row-major
 * (out x in).  The loss is L = (1/(2B)) sum over the batch and both outputs of (y - t)^2.
 *
 * All data pointers are device pointers on the handle's (or the current) device.
 * ------------------------------------------------------------------------------------------ */
typedef struct gw_mlp gw_mlp;

/* Number of parameters of an n_in -> hidden x 3 -> 2 network. */
GW_API gw_status gw_mlp_num_params(int n_in, int hidden, size_t *n);

/* Network with zero parameters and Adam state.
 *   n_in       1..64
 *   hidden     1..1024
 *   max_batch  largest batch of gw_mlp_grad / gw_mlp_train_step, and the chunk of gw_mlp_forward;
 *              1..2^22
 *   stream     cudaStream_t for every call on the handle (NULL = legacy default stream)
 * Device memory: 5 P floats, P halves, 5 max_batch x hidden floats, a split-K workspace of
 * 64 x hidden x (hidden + 1) floats, and the tensor-core operands of training at 6 bytes a value
 * (three BF16 parts): 6 x (7 hidden + 144) bytes per row of max_batch (activations and deltas in
 * two orientations; the inputs padded to 16 and 128) plus five weight matrices; gw_mlp_infer adds
 * 272 KB of tiled weights. */
GW_API gw_status gw_mlp_create(gw_mlp **out, int device, int n_in, int hidden, int max_batch, void *stream);
GW_API gw_status gw_mlp_destroy(gw_mlp *m);
GW_API gw_status gw_mlp_last_error(gw_mlp *m, char *buf, size_t n);

/* Copy the flat parameters in (this resets Adam's moments and step count) or out.  theta is a
 * host pointer (on_device = 0; the call then synchronises) or a device pointer (1). */
GW_API gw_status gw_mlp_set_params(gw_mlp *m, const float *theta, int on_device);
GW_API gw_status gw_mlp_get_params(gw_mlp *m, float *theta, int on_device);

/* Inference: Y[n][2] = network(X[n][n_in]), in chunks of max_batch rows, with the arithmetic of
 * training (FP32 activations; the hidden layers' products on the tensor cores with each FP32
 * operand as three BF16 parts, FP32-accurate). */
GW_API gw_status gw_mlp_forward(gw_mlp *m, const float *X, long n, float *Y);

/* Inference on the tensor cores: the same network with FP16 weights and FP32 accumulation in one
 * kernel on CTA pairs (tcgen05.mma cta_group::2, each CTA holding half of every weight matrix).
 * Layer 1 multiplies the inputs split into FP16 hi and lo parts (x = hi + lo to about 2^-22), so
 * it keeps FP32 accuracy; the outputs of layers 1 and 2 are rounded to FP16 (the operands of the
 * two 256 x 256 products); tanh is the hardware approximation (tanh.approx.f32, relative error
 * about 2^-11); the output layer runs in FP32.  Requires hidden = 256, n_in <= 16 and |X| < 65504
 * (else GW_E_UNSUPPORTED for the first two).  Any n (no chunking: the kernel walks 256-row tiles).
 * Asynchronous; device-side waits are bounded and report through gw_mlp_check.  Y[n][2] as
 * gw_mlp_forward. */
GW_API gw_status gw_mlp_infer(gw_mlp *m, const float *X, long n, float *Y);

/* Synchronise the handle's stream and return the status of its tensor-core kernels. */
GW_API gw_status gw_mlp_check(gw_mlp *m);

/* Loss and gradient of a batch, without an update.
 *   rows    NULL, or batch sample indices into X[.][n_in] and T[.][2] (a minibatch gather)
 *   grad    receives dL/dtheta (P floats, same flat order as the parameters)
 *   loss    receives L (one float)
 * Weights enter as their FP16 values, so the exact gradient is that of the network whose W_l
 * are rounded to FP16. */
GW_API gw_status gw_mlp_grad(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, float *grad,
                             float *loss);

/* One Adam step (Kingma and Ba, 2015) on a batch:
 *     m <- b1 m + (1 - b1) g
 *     v <- b2 v + (1 - b2) g^2
 *     theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * followed by re-rounding of the FP16 weights.
 *   loss_accum  NULL, or a device float to which this batch's L is added. */
GW_API gw_status gw_mlp_train_step(gw_mlp *m, const float *X, const float *T, const int *rows, int batch, double lr,
                                   double beta1, double beta2, double adam_eps, float *loss_accum);

/*
 * Training of the correction network: `epochs` passes of Adam (the rule of gw_mlp_train_step) over
 * minibatches of the rows of X[n][n_in] and T[n][2] (device pointers), drawn without replacement:
 *   pool   the rows 0..n-1, followed by the rows whose feature diag_feature equals 1 (the
 *          diagonal entries of P~ for gw_corr_features, feature 7), ascending, diag_repeat - 1
 *          more times (diag_repeat = 1 or diag_feature < 0: no repeats).  Diagonal entries carry
 *          most of the correction's norm but are 1 in N_g (N_g + 1)/2 of the rows.
 *   order  pass e takes the pool sorted by key(j) = mix(seed * 0x9E3779B97F4A7C15
 *          + (e + 1) * 0xD1B54A32D192ED03 + j) (64-bit wrapping arithmetic, j the pool position,
 *          mix = SplitMix64's output function, ties by position), split into floor(S / batch)
 *          minibatches; the ragged tail of a pass is dropped.
 *   rate   step t of T = epochs floor(S / batch): lr_final + (lr - lr_final)(1 + cos(pi t / T)) / 2.
 * losses[e] (host float[epochs]) receives the mean minibatch loss of pass e.  The device scratch
 * (the pool, its order and the sort keys, about 24 bytes per pool row) is allocated for the call
 * and released before it returns; the call synchronises the handle's stream.
 */
typedef struct gw_corr_train_opts {
    int epochs;                 /* >= 1 */
    int batch;                  /* 1 .. max_batch of the handle */
    double lr, lr_final;        /* > 0, >= 0 */
    double beta1, beta2, adam_eps;
    unsigned long long seed;
    int diag_repeat;            /* >= 1 */
    int diag_feature;           /* < n_in; negative: none */
} gw_corr_train_opts;
GW_API gw_status gw_corr_train(gw_mlp *m, const float *X, const float *T, long n, const gw_corr_train_opts *opts,
                               float *losses);

/* ratio = sum_{c >= nc_keep} sum_v 2/(E_c - E_v) / sum_{c < nc_keep} sum_v 2/(E_c - E_v), in FP64,
 * from device energies E_eV[nv + nc_all] (occupied first, as gw_load_states).  This is the
 * weight of the omitted pairs in Eq. (Pstatic) relative to the kept ones; it needs only the
 * energies of the omitted states, not their orbitals.  nv <= 1024 (else GW_E_INVALID).  Output:
 * one device float. */
GW_API gw_status gw_corr_weight_ratio(const double *E_eV, int nv, int nc_keep, int nc_all, float *ratio,
                                      void *stream);

/* Features of every upper-triangle entry of a truncated P~.
 *   PG       complex64, ng x ng, as written by gw_P_to_G
 *   ng       >= 2
 *   gvec     int32 [ng][3] integer G-vectors in basis order
 *   ratio    device float from gw_corr_weight_ratio
 *   PG_clos  complex64 ng x ng closure estimate from gw_corr_closure, or NULL (features 10, 11 = 0)
 *   X        float [ng (ng + 1)/2][12]
 *   scale    device float, receives s */
GW_API gw_status gw_corr_features(const void *PG, int ng, const int *gvec, int gcut, const float *ratio,
                                  const void *PG_clos, float *X, float *scale, void *stream);

/*
 * Closure estimate of the omitted part of P~ (Sec. 2 band truncation of the sum over c in
 * Eq. Pstatic; Eq. gpsaceP), from the states loaded in ctx (occupied first, then the kept
 * unoccupied ones; n_in in all) and the energies of the omitted unoccupied states only:
 *     dP~(G, G') = [rho_W(G - G') - sum_v W_v sum_{n < n_in} M_vn(G) conj(M_vn(G'))] / (N_r - n_in)
 * with W_v = sum_{omitted c} 2 / (E_v - E_c) (Hartree), rho_W(q) = sum_r e^{-iq.r} sum_v W_v
 * |psi_v(r)|^2 and M_vn(G) = sum_r e^{-iG.r} conj(psi_v(r)) psi_n(r).  It is the mean of the omitted
 * sum over states drawn without preference in the complement of the loaded ones (closure relation:
 * a complete set sums to the identity on the grid), and exact when the omitted states complete the
 * set and share one energy.  The projector term is a rank nv n_in update on the 16-bit tensor
 * cores (FP16X3, the context's window); rho_W and its whole-grid transform are FP64.
 *   gcut       sphere cut as gw_P_to_G (the sphere is rebuilt if it differs)
 *   E_omit_eV  host double [nc_omit], each above every occupied energy (else GW_E_INVALID)
 *   out        device complex64 [N_g][N_g] (overwritten; Hermitian, zero G = 0 row and column)
 * Uses the context's g-space workspaces (not P~); synchronises the stream.  GW_E_INVALID if the
 * loaded states already span the grid, GW_E_UNSUPPORTED where the grid needs the row-block
 * transform kernel. */
GW_API gw_status gw_corr_closure(gw_ctx *ctx, int gcut, const double *E_omit_eV, int nc_omit, void *out);

/* Training targets T[t][2] = s (P~_all - P~_keep - dP~)(g, h), with s from gw_corr_features on
 * P~_keep and dP~ the closure estimate PG_clos (NULL = 0). */
GW_API gw_status gw_corr_targets(const void *PG_keep, const void *PG_all, const void *PG_clos, int ng,
                                 const float *scale, float *T, void *stream);

/* In place, P~(g,h) += dP~(g,h) + (y0 + i y1)/s and P~(h,g) = its conjugate, for g < h, with dP~
 * the closure estimate PG_clos (NULL = 0).  The diagonal takes the real part only.  Row and
 * column 0 are left unchanged: they vanish exactly at any N_c, because occupied and unoccupied
 * states are orthogonal.
 *   Y  float [ng (ng + 1)/2][2], from gw_mlp_forward */
GW_API gw_status gw_corr_apply(void *PG, int ng, const float *Y, const float *scale, const void *PG_clos,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GW_H */
