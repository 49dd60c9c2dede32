/* collapse.h -- C-ABI of libcollapse, the GB300 (sm_103a) collapse-time library.
 *
 * What it computes (Lepinzan et al., arXiv:2510.02873, Sec. 3 and Sec. 4.1):
 * for every grid point p and smoothing radius r, from the six independent
 * components of the Hessian of the smoothed potential H[r][c][p]
 * (c = xx, yy, zz, xy, xz, yz):
 *   1. the eigenvalues l1 >= l2 >= l3 of the symmetric 3x3 matrix (Sec. 3);
 *   2. the growth factor at collapse D_c, the smallest positive root of the
 *      third-order LPT stretch of axis 1 (Sec. 3, "Classic" collapse time):
 *        A_1(D) = 1 - D l1 - 3/7 D^2 l2 l3 + D^3 [l1 l2 l3/9 - 5/21 l1 (l2^2 + l3^2)];
 *      l1 <= 0, or D_c beyond the last table entry: no collapse, F = 0;
 *   3. the collapse scale factor a_c = a(D_c) from a natural cubic spline of
 *      the inverse growth function through (D(a_k), a_k), D(a) being the
 *      solution of the linear growth ODE (Sec. 3; spline built once, Sec. 4.2);
 *      below the first knot a_c = a_0 D_c / D(a_0);
 *   4. F = 1/a_c = 1 + z_c, and the per-point running maxima
 *      "F_max[p] = F, idx[p] = r if F > F_max[p]" (Sec. 4.1: read/modify/write
 *      of two output arrays; ties keep the earlier radius).
 *
 * Conventions for every call:
 *   - Device pointers are caller-owned (e.g. torch tensors); the library never
 *     frees them and keeps no reference after the call returns. Host pointers
 *     are read or written during the call only.
 *   - All device work is enqueued on the caller's stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream); calls do not
 *     synchronise unless stated.
 *   - Return value: CC_OK (0) or a CC_E* code; no exceptions, no exit().
 *     cc_strerror() names the code; cc_last_error_message() gives detail.
 *   - One context per device; a context is not thread-safe (serialise calls
 *     on one context, or use one context per host thread). Device work of
 *     calls on one context that use its workspaces (CC_MODE_MIXED, which
 *     keeps records of the points with FP64-heavy radii between its two
 *     kernels; cc_collapse_multi_host; the surrogate's training) must not
 *     overlap on the GPU: enqueue them on one stream or order the streams.
 *     CC_MODE_MIXED allocates that workspace on first use at a size (24 B
 *     per record, for at most n (0.006 R + 0.02) + 1024 records, R capped at
 *     256): the first call at a new size is not asynchronous.
 *   - F_max/idx entries hold what cc_reset_max or an earlier collapse call
 *     left (F_max >= 0; idx = -1, or a scale index >= 0).
 *   - Supported input range: eigenvalue magnitudes of H up to 1e6 (in units
 *     where D(a = 1) = 1; collapse needs at least ~0.7, and points with l1 <= 0
 *     never collapse). The FP32 seeds of every path form sixth powers of the
 *     eigenvalues, which leave the FP32 range near 2.6e6; beyond 1e6 results
 *     are not guaranteed. Non-finite components give no collapse (F = 0).
 *   - Plane layout: component c of point p at radius r is
 *       hess[r * radius_stride + c * plane_stride + p]   (elements, not bytes);
 *     plane_stride >= n, radius_stride >= 6 * plane_stride. Each plane must
 *     start on a 16-byte boundary (so plane_stride * elem_size and
 *     radius_stride * elem_size are multiples of 16 and hess is 16-byte
 *     aligned); other layouts return CC_EINVAL.
 */
#ifndef COLLAPSE_H
#define COLLAPSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CC_API __attribute__((visibility("default")))
#else
#define CC_API
#endif

/* ---- status codes ---- */
#define CC_OK        0
#define CC_EINVAL    1  /* bad argument (null pointer, size, stride, alignment, mode) */
#define CC_ECUDA     2  /* a CUDA runtime call failed (detail in cc_last_error_message) */
#define CC_ENOMEM    3  /* device or host allocation failed */
#define CC_ETIMEOUT  4  /* a bounded device-side wait gave up (persistent kernels) */
#define CC_ERANGE    5  /* input outside the supported range (e.g. table bounds) */
#define CC_ENOTSUP   6  /* mode or dtype not available in this build */

/* ---- element types of the Hessian planes ---- */
#define CC_F64 8
#define CC_F32 4

/* ---- evaluation modes ---- */
typedef enum {
  CC_MODE_FP64 = 0,     /* FP64 path (Sec. 3 "Classic" kernel): FP64 invariants, Newton
                         * corrections and spline, FP32 seeds; F within 1e-10 relative   */
  CC_MODE_MIXED = 1,    /* FP32 bulk, FP64 for the sensitive branches                   */
  CC_MODE_SURROGATE = 2,/* learned surrogate with exact fallback                        */
  CC_MODE_TABULATED = 3,/* table of 1/D_c in (delta, x, y) (Sec. 3 "Tabulated" kernel)   */
  CC_MODE_F32X2 = 4,    /* the FP64 path's steps in float-float arithmetic (pairs of FP32
                         * numbers, 48 significant bits) instead of the FP64 unit; same
                         * accuracy contract as CC_MODE_FP64 (F within 1e-10 relative)     */
  CC_MODE_EXACT_GROWTH = 5 /* FP64 path with the EdS growth ratios of the collapse condition
                         * replaced by the second- and third-order growth factors of the
                         * context's background (D2/D1^2, D3a/D1^3, D3b/D1^3 as splines in D) */
} cc_mode;

/* Flat LCDM-like background: E^2 = Om a^-3 + (1 - Om - OL) a^-2 + OL.
 * n_knots log-spaced scale factors in [a_min, a_max] (2 <= n_knots <= 4096,
 * 1e-5 < a_min < a_max); D is normalised to D(a = 1) = 1. The device tables
 * (cc_create, cc_collapse_multi_noalloc) also need D to at most double between
 * neighbouring knots (n_knots >= 11 for a_max / a_min = 1000; the paper's 512
 * knots give 1.3 %); coarser tables return CC_EINVAL. */
typedef struct {
  double omega_m;
  double omega_l;
  int32_t n_knots;
  double a_min;
  double a_max;
} cc_cosmology;

typedef struct cc_ctx cc_ctx;

/* Device-side counters accumulated by every collapse launch since the last
 * cc_reset_stats (read with cc_get_stats, which synchronises the stream). */
typedef struct {
  uint64_t evaluations;   /* (point, radius) evaluations                                   */
  uint64_t collapsed;     /* evaluations with F > 0                                         */
  uint64_t eds_branch;    /* D_c below the first knot (a_c = a_0 D_c / D_0)                 */
  uint64_t refined;       /* eigenvalue pairs re-solved by deflation (near-degenerate pair) */
  uint64_t fp64_branch;   /* MIXED: points re-evaluated in FP64                             */
  uint64_t fallback;      /* SURROGATE: points sent to the exact path                       */
  uint32_t error_flags;   /* device-side error bits: 1 = a bounded wait for tensor-core
                           * completion ran out in the CC_SURROGATE_TCGEN05 kernel (that
                           * launch's results are incomplete); 2 = (library built with
                           * CC_DEBUG only) a table index left its range and was
                           * clamped; 0 otherwise                                             */
  uint32_t reserved;
} cc_stats;

/* Create a context on `device`: solves the growth ODE in FP64 on the host,
 * builds the natural spline of a(D) and uploads it once (Sec. 3, Sec. 4.2),
 * with its float-float image (CC_MODE_F32X2) and the second- and third-order
 * growth-ratio splines (CC_MODE_EXACT_GROWTH). Allocates device memory for
 * the tables and counters. */
CC_API int cc_create(cc_ctx **out, const cc_cosmology *cosmo, int device);

/* Release the context and its device memory (synchronises the device). NULL is a no-op. */
CC_API void cc_destroy(cc_ctx *ctx);

/* Host only (no device needed): the library's growth table for `cosmo`,
 * a_k and D_k with cosmo->n_knots entries each (Sec. 3: D(a) from its ODE). */
CC_API int cc_build_growth_table(const cc_cosmology *cosmo, double *a_k, double *D_k);

/* Host copies of the library's growth table: a_k and D_k (n = n_knots entries each). */
CC_API int cc_get_growth_table(const cc_ctx *ctx, double *a_k, double *D_k, int32_t n);

/* F_max[p] = 0 and idx[p] = -1 for p < n (Sec. 4.1: device array initialisation). */
CC_API int cc_reset_max(cc_ctx *ctx, double *F_max, int32_t *idx, int64_t n, void *stream);

/* One smoothing radius: evaluates F for n points of one radius and applies the
 * running-maximum update with index scale_idx (Sec. 4.1).
 *   hess: device, 6 planes (layout above), dtype CC_F64 or CC_F32;
 *   sigma_R: rms of tr H at this radius; used only by MIXED (degeneracy
 *            threshold) and SURROGATE (input normalisation), must be > 0;
 *   F_max (FP64), idx (int32): device, n entries, updated in place. */
CC_API int cc_collapse_scale(cc_ctx *ctx, cc_mode mode, const void *hess, int32_t dtype, int64_t n,
                      int64_t plane_stride, double sigma_R, double *F_max, int32_t *idx,
                      int32_t scale_idx, void *stream);

/* R radii in one launch, equivalent to R calls of cc_collapse_scale with
 * scale indices scale_idx0 .. scale_idx0 + R - 1 in that order; the running
 * maximum is kept in registers and F_max/idx are read and written once.
 *   sigma: host array of R values (> 0). */
CC_API int cc_collapse_multi(cc_ctx *ctx, cc_mode mode, const void *hess, int32_t dtype, int64_t n,
                      int64_t plane_stride, int64_t radius_stride, const double *sigma, int32_t R,
                      double *F_max, int32_t *idx, int32_t scale_idx0, void *stream);

/* Host-resident variant of cc_collapse_multi (the paper's workflow copies the
 * Hessian planes to the device for every radius, Sec. 3 and Sec. 5.6):
 * hess_host, F_max_host and idx_host are HOST pointers (page-locked memory
 * gives copy/compute overlap; pageable memory works, slower). Radius planes
 * are copied into a device double buffer on a copy stream while the previous
 * radius is evaluated on `stream`; F_max/idx are copied in, updated on the
 * device and copied back. Blocks until the host outputs are written.
 * Device staging memory (2 radii of planes + outputs) is allocated on first
 * use, grown when needed and kept by the context until cc_destroy. */
CC_API int cc_collapse_multi_host(cc_ctx *ctx, cc_mode mode, const void *hess_host, int32_t dtype,
                           int64_t n, int64_t plane_stride, int64_t radius_stride,
                           const double *sigma, int32_t R, double *F_max_host, int32_t *idx_host,
                           int32_t scale_idx0, void *stream);

/* No counterpart in the paper. A variant of cc_collapse_multi for callers that
 * cannot allocate device memory (code whose device memory is owned by another
 * framework's caching allocator, or loops that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree). It needs no context and makes no
 * allocation of any kind: the spline table for `cosmo` and the launch counters
 * live in a file-scope static device array of 53.5 KB that every GPU loading
 * the library holds until exit. Inputs and outputs are the caller's device
 * buffers, as for cc_collapse_multi (same layout rules and results).
 *   cosmo: host; n_knots must be <= 1024, larger tables return CC_EINVAL.
 *   mode: CC_MODE_FP64 only (others return CC_ENOTSUP).
 *   stats: host, may be NULL; when given, receives this call's counters and
 *          the call synchronises `stream`.
 * All calls on a device share the array and it keeps the last call's contents:
 * the counters are cleared at the start of each call, and the table is copied
 * in again when the cosmology changes. Calls that overlap on the GPU (other
 * streams, or another cosmology in flight) race on it. The first call on each
 * device looks up the array's address (with that device current) and uploads
 * the table. */
CC_API int cc_collapse_multi_noalloc(const cc_cosmology *cosmo, cc_mode mode, const void *hess,
                              int32_t dtype, int64_t n, int64_t plane_stride,
                              int64_t radius_stride, const double *sigma, int32_t R,
                              double *F_max, int32_t *idx, int32_t scale_idx0, cc_stats *stats,
                              void *stream);

/* ---- tabulated collapse and the interpolation routines (Sec. 3, 4.2, 4.3) ----
 * The "Tabulated" option precomputes collapse times on a grid of
 * delta = l1 + l2 + l3, x = l1 - l2, y = l2 - l3 and interpolates with a cubic
 * spline along delta and bilinear interpolation in x and y (Sec. 3, Sec. 4.2).
 * The tabulated quantity here is u = 1/D_c (the inverse growth factor at
 * collapse: finite everywhere, nearly linear in (delta, x, y)).
 *   dgrid (nd, 4..256), xgrid (nx, 2..256), ygrid (ny, 2..256): host, strictly
 *   increasing, x and y axes starting at >= 0;
 *   values: host, nx * ny * nd, values[(ix * ny + iy) * nd + k] = u(d_k, x_ix, y_iy). */

/* Copy a table to the context and build its natural splines along delta on the
 * device (the paper rebuilds them at every smoothing radius, Sec. 4.2). Later
 * CC_MODE_TABULATED launches use it; points outside [d_0, d_last] x [x_0, x_last]
 * x [y_0, y_last] (the first and last knot of each axis) fall back to the
 * R-LPT root. Device memory for the table is
 * allocated on first use and kept by the context. Calls on one context are
 * stream-ordered: do not replace a table that launches on another stream still read. */
CC_API int cc_set_table(cc_ctx *ctx, const double *dgrid, int32_t nd, const double *xgrid, int32_t nx,
                        const double *ygrid, int32_t ny, const double *values, void *stream);

/* Helper for building a table without an external collapse model: u = 1/D_c of
 * the R-LPT condition at every node, computed on the device; values (host) receives
 * nx * ny * nd entries in the layout above. Synchronises `stream`. */
CC_API int cc_table_nodes_rlpt(cc_ctx *ctx, const double *dgrid, int32_t nd, const double *xgrid, int32_t nx,
                               const double *ygrid, int32_t ny, double *values, void *stream);

/* The table interpolation routine on its own (the paper's spline x bilinear
 * toy, Sec. 4.3): out[i] = u(d[i], x[i], y[i]) for m device queries; outside the
 * axes the edge cells extrapolate. */
CC_API int cc_table_query(cc_ctx *ctx, const double *d, const double *x, const double *y, int64_t m,
                          double *out, void *stream);

/* The cubic-spline routine on its own (the paper's y(x) toy, Sec. 4.3): a
 * natural cubic spline through n host knots (2 <= n <= 4096, strictly
 * increasing xk), built on the host in FP64 (one O(n) tridiagonal solve) and
 * uploaded with the call, evaluated on the device at m device queries q into
 * out (device); outside the knots the end intervals extrapolate. */
CC_API int cc_spline_eval(cc_ctx *ctx, const double *xk, const double *yk, int32_t n, const double *q,
                          int64_t m, double *out, void *stream);

/* ---- learned surrogate (no counterpart in the paper) ----
 * An MLP 3 -> 64 -> 64 -> 64 -> 1 (SiLU) maps z = (l1, l2, l3) / s(R) to
 * f ~ log(D_c s(R)). CC_MODE_SURROGATE uses f only to seed the Newton iteration
 * of the collapse condition (FP32 eigenvalues as in CC_MODE_MIXED); a point is
 * accepted when the last Newton step is below 1e-6 D and z lies inside the
 * training hull, otherwise it takes the exact FP64 path (counted in
 * cc_stats.fallback). Accuracy is that of CC_MODE_MIXED (3e-5 on F). */
typedef struct {
  int32_t steps;        /* Adam steps (>= 1) */
  int32_t batch;        /* samples per step, a multiple of 64 */
  float lr;             /* peak learning rate (warm-up 100 steps, cosine decay) */
  uint64_t seed;        /* initial weights and minibatch sampling */
  float val_fraction;   /* held-out share of the samples, in (0, 0.5) */
} cc_train_config;

typedef struct {
  int64_t samples, train_samples, val_samples;  /* collapsing points used */
  float loss_first, loss_last;                  /* minibatch MSE of log(D_c s) */
  float val_rms, val_max;                       /* held-out |f - log(D_c s)| */
  float hull_lo[3], hull_hi[3];                 /* training range of z */
} cc_train_report;

/* Train the context's surrogate on the GPU (BF16 tensor-core forward and
 * backward, FP32 accumulation, FP32 Adam). Targets come from the exact FP64
 * path on the given Hessian planes (device, 6 planes of n points, dtype
 * CC_F64/CC_F32) at rms s = sigma: every point with l1 > 0 and D_c s < 1e4 is a
 * sample. Allocates device memory for the samples (16 B per point) and the
 * network, kept by the context. Synchronises `stream`. */
CC_API int cc_surrogate_train(cc_ctx *ctx, const void *hess, int32_t dtype, int64_t n, int64_t plane_stride,
                              double sigma, const cc_train_config *cfg, cc_train_report *report, void *stream);

/* Parameters (8641 floats: W1[3][64], b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4)
 * and hull (lo[3], hi[3]) of the current surrogate, to host memory. */
CC_API int cc_surrogate_params(const cc_ctx *ctx, float *params, float *hull);

/* Install a surrogate from host parameters and hull (layout as above). It
 * carries no optimiser state: training cannot resume from it (use a checkpoint). */
CC_API int cc_load_surrogate(cc_ctx *ctx, const float *params, const float *hull);

/* Checkpoint of the training state (no counterpart in the paper): a versioned
 * host blob holding the schedule (seed, learning rate, batch, held-out share,
 * length of the learning-rate schedule), the Adam step count, the hull, and
 * the FP32 parameters with both Adam moments. The minibatch sampler is
 * counter-based (indices hashed from the seed and the step), so the step is
 * its whole state.
 *   cc_surrogate_checkpoint: blob NULL -> *bytes receives the size; otherwise
 *     *bytes >= that size, the blob is written and *bytes set to its size.
 *     CC_EINVAL before any training (or after cc_load_surrogate).
 *   cc_surrogate_restore: installs a blob written by cc_surrogate_checkpoint
 *     (any context, any device); CC_EINVAL for a blob that is not one, of
 *     another size or with values out of range, CC_ENOTSUP for another version.
 *   cc_surrogate_train_resume: continues training from the context's state
 *     (after cc_surrogate_train or cc_surrogate_restore) for `steps` more Adam
 *     steps on samples of the given planes (rebuilt as in cc_surrogate_train);
 *     the learning rate follows the warm-up + cosine schedule of length
 *     schedule_steps (0: the stored length, extended to cover the new steps).
 *     The hull becomes the union of the stored one and the new samples'.
 *     Synchronises `stream`. */
CC_API int cc_surrogate_checkpoint(const cc_ctx *ctx, void *blob, size_t *bytes);
CC_API int cc_surrogate_restore(cc_ctx *ctx, const void *blob, size_t bytes);
CC_API int cc_surrogate_train_resume(cc_ctx *ctx, const void *hess, int32_t dtype, int64_t n, int64_t plane_stride,
                                     double sigma, int32_t steps, int32_t schedule_steps, cc_train_report *report,
                                     void *stream);

/* Kernel that runs CC_MODE_SURROGATE. Both evaluate the same network with
 * BF16 operands and FP32 accumulation, and both results meet the mixed path's
 * tolerance; they differ in how the MMAs are issued:
 *   CC_SURROGATE_TCGEN05 (default): fifth-generation tensor cores; groups of
 *     128 threads each own an M = 128 tile of points, accumulators in tensor
 *     memory, eight groups per CTA (one CTA per SM) sharing weights staged by
 *     one bulk copy, each layer's bias carried by two extra K columns;
 *   CC_SURROGATE_MMA_SYNC: warp-level mma.sync m16n8k16, 32 points per warp
 *     as two 16-row tiles, activations chained in registers.
 * Returns CC_EINVAL for another value. */
typedef enum { CC_SURROGATE_MMA_SYNC = 0, CC_SURROGATE_TCGEN05 = 1 } cc_surrogate_engine;
CC_API int cc_set_surrogate_engine(cc_ctx *ctx, int32_t engine);

/* f(z) for n device inputs z (n x 3) into out (device), on the tensor-core path. */
CC_API int cc_surrogate_eval(cc_ctx *ctx, const float *z, int64_t n, float *out, void *stream);

/* One minibatch of the training kernel on host samples (n a multiple of 64):
 * gradient of mean (f(z_i) - t_i)^2 into grad (host, 8641) and the loss.
 * Synchronises the device. For checking the training kernels. */
CC_API int cc_surrogate_grad(cc_ctx *ctx, const float *z, const float *t, int32_t n, float *grad, float *loss);

/* ---- batches of independent realizations (one persistent launch) ----
 * Many realizations of uneven grid sizes and radius counts (e.g. a set of
 * simulation boxes) are evaluated by ONE persistent kernel: its CTAs take
 * tiles of points from a device work counter until every tile of every
 * realization is done, each tile running all radii of its realization with
 * the running maximum in registers (the per-point work of Sec. 4.1). */
typedef struct {
  const void *hess;       /* device planes of this realization (layout as cc_collapse_multi) */
  int32_t dtype;          /* CC_F64 or CC_F32 */
  int64_t n;              /* points */
  int64_t plane_stride;   /* elements between component planes (16-byte aligned planes) */
  int64_t radius_stride;  /* elements between radii */
  int32_t R;              /* radii, 1..256 */
  const double *sigma;    /* host, R values > 0 (copied at cc_batch_create) */
  double *F_max;          /* device, n entries, updated in place */
  int32_t *idx;           /* device, n entries, updated in place */
  int32_t scale_idx0;     /* index of this realization's first radius */
} cc_batch_item;

typedef struct cc_batch cc_batch;

/* Validate the items and build a plan: the item table, per-radius parameters
 * and a work counter are copied to device memory owned by the plan (allocated
 * here). The device buffers the items point to must outlive the plan.
 * CC_MODE_MIXED plans also own the record buffer for the points with
 * FP64-heavy radii (24 B per record, for at most sum_i n_i (0.006 R_i + 0.02)
 * + 1024 records), so runs of one plan must not overlap on the GPU. Limits:
 * nitems < 2^23, n < 2^40 per item. */
CC_API int cc_batch_create(cc_ctx *ctx, cc_mode mode, const cc_batch_item *items, int32_t nitems,
                           cc_batch **out);

/* Autotuner: per size class (realizations grouped by ceil(log2 n)) picks the
 * points per tile, and for the whole batch the threads per block, by timing
 * candidate launches on the class's own realizations (this runs the kernel and
 * therefore updates their F_max/idx; reset them afterwards). With cache_path
 * non-NULL, choices are read from / appended to that text file, keyed by GPU
 * name, mode and class. Synchronises `stream`. */
CC_API int cc_batch_autotune(cc_batch *b, const char *cache_path, void *stream);

/* One persistent launch over all items on `stream` (work-counter reset + kernel;
 * CC_MODE_MIXED: then the record-counter reset and two kernels for the
 * recorded points). */
CC_API int cc_batch_run(cc_batch *b, void *stream);

/* The same launch through a CUDA graph that the plan captures on first use
 * (on `stream`, which must not be capturing) and replays afterwards. */
CC_API int cc_batch_run_graph(cc_batch *b, void *stream);

/* Chosen shape: threads per block, and points per tile for each item. */
CC_API int cc_batch_get_config(const cc_batch *b, int32_t *threads_per_block, int32_t *tile_points,
                               int32_t nitems);

CC_API void cc_batch_destroy(cc_batch *b);

/* Counts of F_max per bin: the number of collapsed points per redshift bin
 * of the paper's production-run check (Sec. 5.5), with F = 1 + z_c.
 *   F_max  device, n values >= 0 (as written by the collapse calls; 0 = no collapse)
 *   edges  host, nbins + 1 values, positive, finite, strictly increasing (1 <= nbins <= 1023)
 *   counts device, nbins + 2 values, overwritten (asynchronously on `stream`):
 *          counts[0] = #{F < edges[0]} (every non-collapsed point among them),
 *          counts[1 + k] = #{edges[k] <= F < edges[k + 1]},
 *          counts[nbins + 1] = #{F >= edges[nbins]}.
 * Integer work: exact, independent of the order of the points. Errors:
 * CC_EINVAL for bad edges, NULL or misaligned (8-byte) pointers. */
CC_API int cc_histogram(cc_ctx *ctx, const double *F_max, int64_t n, const double *edges, int32_t nbins,
                        unsigned long long *counts, void *stream);

/* ---- device-resident field -> smoothed Hessian planes ------------------
 * The FFT stage ahead of the collapse computation (Sec. 3: PINOCCHIO's FFTs
 * produce the second derivatives of the potential; keeping them on the device
 * between the FFTs and the collapse kernel is the step the paper plans).
 * Conventions: an N^3 periodic grid of side `box`, cells in C order (x
 * slowest, z fastest); wavenumbers k = 2 pi m / box (m the signed DFT
 * frequency); delta_k = DFT(w) sqrt(P(k)) for unit white noise w, with
 * P(k) = amplitude k^index exp(-(k / k_cut)^2), Nyquist modes (any |m| = N/2)
 * and k = 0 zeroed, so var(delta) = mean of P over the k grid; the Hessian at
 * radius R is H_ij = IDFT[(k_i k_j / k^2) exp(-k^2 R^2 / 2) delta_k] (its trace
 * is the smoothed density). The transforms are cuFFT's. */
typedef struct {
  double box;        /* side of the periodic box (same length unit as R) */
  double amplitude;  /* A of P(k) = A k^index exp(-(k/k_cut)^2), > 0 */
  double index;
  double k_cut;      /* > 0 */
} cc_spectrum;

typedef struct cc_field cc_field;

/* Colours the unit white noise `white` (device, N^3 doubles, C order,
 * 16-byte aligned; not modified) into delta_k, kept on the device by the field
 * (N even, 4 <= N <= 1024). Synchronises `stream` once. */
CC_API int cc_field_create(cc_ctx *ctx, const double *white, int32_t N, const cc_spectrum *spec, cc_field **out,
                           void *stream);

/* rms of the density smoothed at radius R, sqrt(mean over the k grid of
 * P(k) exp(-k^2 R^2)) (the s(R) to pass with the planes); synchronises. */
CC_API int cc_field_sigma(cc_field *f, double R, double *sigma, void *stream);

/* The six Hessian planes at radius R (components xx yy zz xy xz yz, each N^3
 * values in C order, plane c at planes + c * plane_stride elements) in FP64
 * (dtype CC_F64) or FP32 (CC_F32: FP32 inverse transforms of the FP64 k-space
 * products). plane_stride >= N^3, planes 16-byte aligned. Asynchronous on
 * `stream`; the first call for a (dtype, plane_stride) pair builds a cuFFT plan. */
CC_API int cc_field_hessian(cc_field *f, double R, void *planes, int32_t dtype, int64_t plane_stride, void *stream);

CC_API void cc_field_destroy(cc_field *f);

/* Counters since the last reset (synchronises `stream`). */
CC_API int cc_get_stats(cc_ctx *ctx, cc_stats *out, void *stream);
CC_API int cc_reset_stats(cc_ctx *ctx, void *stream);

/* Names of status codes and the detail of the last error on this thread. */
CC_API const char *cc_strerror(int code);
CC_API const char *cc_last_error_message(void);

/* Library version as major*10000 + minor*100 + patch. */
CC_API int cc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* COLLAPSE_H */
