/*
 * mlens.h -- C ABI of libmlens, a GB300 (sm_103a) backward ray-shooter for
 * gravitational microlensing by a random star field.
 *
 * The method (arXiv:1703.09707, Section 1 and Section 2.2):
 *   Eq. (3)      alpha(theta) = [[kc+g1, g2], [g2, kc-g1]] theta
 *                               + sum_i m_i (theta - theta_i) / |theta - theta_i|^2
 *   Eq. (2)      beta = theta - alpha
 *   Algorithm 1  for every ray theta_ij of a uniform lens-plane grid: compute
 *                alpha and beta, convert beta to source-pixel coordinates and
 *                add one to mag[j_s][i_s] when the pixel is in the window.
 * Angles are in Einstein radii of a 1 M_sun lens and masses in M_sun (Eq. 4).
 *
 * Conventions shared by every entry point
 *   - Status: 0 (MLENS_OK) on success, a negative MLENS_ERR_* code otherwise;
 *     mlens_last_error() returns a message for the calling thread's last
 *     failure.  No C++ exception crosses this boundary.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees them.  Pointers named *_host are ordinary host memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued asynchronously on it; a call returns before the GPU finishes
 *     unless it says otherwise (any call given a non-NULL stats_host waits for
 *     the stream, because the counters are read back).
 *   - Ray grids and source maps are mlens_grid boxes [x0,x1) x [y0,y1) cut into
 *     nx x ny cells.  Rays sit at cell centres:
 *         theta_x(i) = x0 + (i + 1/2) (x1 - x0) / nx,  0 <= i < nx (same for y).
 *     The source pixel of beta is floor((beta_x - x0) * nx / (x1 - x0)) (same
 *     for y), lower edge inclusive, upper edge exclusive.  Counts are uint32,
 *     row-major, row = y pixel: counts[j_s * nx + i_s] (mag[j_s, i_s] of
 *     Algorithm 1).  A ray with a non-finite beta (a ray exactly on a star) is
 *     not binned and is counted in rays_nan; a finite beta outside the window
 *     is counted in rays_out.
 *   - Star coordinates and masses are stored as float32 on the device (the
 *     double inputs are rounded once); every precision variant, FP64 included,
 *     works on those rounded values.
 */
#ifndef MLENS_H
#define MLENS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MLENS_OK               0
#define MLENS_ERR_ARG         -1  /* invalid argument: NULL pointer, bad size, non-finite value */
#define MLENS_ERR_CUDA        -2  /* a CUDA runtime call or a launch failed */
#define MLENS_ERR_NOMEM       -3  /* a device allocation failed */
#define MLENS_ERR_STATE       -4  /* the call is not valid in the context's current state */
#define MLENS_ERR_UNSUPPORTED -5  /* no usable sm_103a device, or an option the library lacks */

/* ------------------------------------------------------ precision variants */
/* FP32 direct sum with star and ray coordinates re-centred on each ray tile,
 * plain FP32 accumulation inside chunks of 32 stars and Kahan-compensated
 * addition of the chunk partials; beta carried as an unevaluated float pair
 * and binned exactly.  The default. */
#define MLENS_PREC_FP32        0
/* FP32 with absolute coordinates and one running FP32 sum per component
 * (the textbook single-precision loop; kept to show its error). */
#define MLENS_PREC_FP32_NAIVE  1
/* IEEE FP64 with the operations in the order of Eq. (3) and stars in input
 * order; its beta and maps equal the FP64 oracle's bit for bit. */
#define MLENS_PREC_FP64        2

/* ---------------------------------------------------------- shoot flags */
#define MLENS_ACCUMULATE 1u       /* add into counts_dev instead of overwriting it */

typedef struct mlens_ctx mlens_ctx;

/* Box [x0,x1) x [y0,y1) cut into nx x ny cells (a ray grid or a source map). */
typedef struct {
    double x0, x1, y0, y1;
    int32_t nx, ny;
} mlens_grid;

/* Ray bookkeeping of one call: rays_total = rays_binned + rays_out + rays_nan. */
typedef struct {
    uint64_t rays_total, rays_binned, rays_out, rays_nan;
} mlens_stats;

/*
 * mlens_create -- upload one star field and the smooth lens terms of Eq. (1).
 * Section 2.2: the star field is generated on the host and copied to the
 * accelerator once.
 *   out        receives the new context (set to NULL on failure).
 *   xy_host    n x 2 star positions (x0, y0, x1, y1, ...), finite, |x|,|y| < 1e12.
 *   m_host     n masses, finite, >= 0.
 *   n          number of stars, 0 <= n < 2^31 (n = 0 is a pure kappa/gamma sheet).
 *   kappa_c, gamma1, gamma2   smooth convergence and external shear (finite).
 *   precision  one of MLENS_PREC_*.
 * Allocates device memory on the current CUDA device (about 16 bytes per star
 * plus a few hundred bytes) and synchronises that device.  The context is tied
 * to that device; use it from one host thread at a time.
 * Errors: MLENS_ERR_ARG, MLENS_ERR_NOMEM, MLENS_ERR_UNSUPPORTED, MLENS_ERR_CUDA.
 */
int mlens_create(mlens_ctx **out, const double *xy_host, const double *m_host, int64_t n,
                 double kappa_c, double gamma1, double gamma2, int32_t precision);

/* Choose the precision variant used by later calls on this context. */
int mlens_set_precision(mlens_ctx *ctx, int32_t precision);

/*
 * mlens_set_tuning -- launch shape of the FP32 kernels for later calls on this
 * context: rays_per_thread in {4, 8} (tile 64 x 16 or 64 x 32 rays per CTA of
 * 256 threads), star_stage in {128, 256, 512} stars staged through shared
 * memory at a time (0 = 256), and fma_pairs in {0, 1}: 0 takes every
 * reciprocal 1/r^2 from the MUFU unit (16 per SM per clock, the bound of the
 * direct sum); 1 takes a share of them (a thread's first ray pair on every third
 * star, 7.8 %) from Newton-Raphson iterations on the FMA pipe instead, which
 * balances the two units (4.84e12 against 4.67e12 interactions/s on GB300).  The
 * stage size never changes the arithmetic; the tile shape (it moves the tile
 * centres) and the reciprocal source change beta in its last bits (never by
 * more than the error bar).  A given setting is deterministic.  Defaults: 8,
 * 256, 1.
 */
int mlens_set_tuning(mlens_ctx *ctx, int32_t rays_per_thread, int32_t star_stage, int32_t fma_pairs);

/*
 * mlens_set_star_split -- how many CTAs share one ray tile's star sum in the
 * FP32 re-centred kernel (MLENS_PREC_FP32 with the default 256-star stage, with
 * either fma_pairs; other settings never split).  The paper's closing discussion
 * of very large star fields proposes splitting the bending-angle sum of one
 * image position over several threads; here each of `split` CTAs sums one of
 * `split` consecutive 32-star-aligned slices of the stars with the same
 * compensated loop, and the slices' partial sums are folded in slice order
 * before beta and binning.  split = 2 .. 8: the CTAs form a thread-block
 * cluster and the first folds the others' partials, read through distributed
 * shared memory.  split = 9 .. 4096: each CTA stores its partials in global
 * memory (a context workspace of up to 256 MB, allocated on first use and kept
 * until mlens_destroy; tile rows are taken in passes that fit it) and a second
 * kernel folds them per tile.  That keeps the GPU full when a grid has few tiles
 * for its star count.  split = 1 never splits; 0 (the default) chooses per call
 * from the number of tiles, the SM count and the star count (at least 2048
 * stars per slice).  The sum's order depends on the split, so beta may differ in
 * its last bits between splits (never by more than the error bar); a given split
 * is deterministic.  Errors: MLENS_ERR_ARG; MLENS_ERR_NOMEM if the workspace
 * cannot be allocated (at the shoot call).
 */
int mlens_set_star_split(mlens_ctx *ctx, int32_t split);

/*
 * mlens_star_split_for -- the split mlens_shoot / mlens_shoot_beta will use on
 * this context for the ray grid `rays` (1 = none).  Errors: MLENS_ERR_ARG.
 */
int mlens_star_split_for(const mlens_ctx *ctx, const mlens_grid *rays, int32_t *split_out);

/*
 * mlens_shoot -- Algorithm 1 over a whole ray grid: deflect every ray by Eq. (3),
 * map it to the source plane by Eq. (2) and count it in its source pixel.
 *   rays       ray grid; 1 <= nx, ny <= 2^20 and nx*ny <= 2^40.
 *   src        source map; 1 <= nx, ny and nx*ny <= 2^30.
 *   counts_dev src.ny x src.nx uint32, device, caller-owned, 4-byte aligned.
 *              Overwritten (zeroed first, on the stream) unless flags has
 *              MLENS_ACCUMULATE.  Counts do not saturate: a pixel past 2^32-1
 *              rays wraps (never reached at the ray densities of the paper).
 *   flags      0 or MLENS_ACCUMULATE.
 *   stats_host optional; when non-NULL the call waits for the stream and fills it.
 *   stream     cudaStream_t or NULL.
 * Errors: MLENS_ERR_ARG (bad grid, NULL counts), MLENS_ERR_CUDA.
 */
int mlens_shoot(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                uint32_t flags, mlens_stats *stats_host, void *stream);

/*
 * mlens_shoot_beta -- mlens_shoot that also writes every ray's source position,
 * for verification.  beta_dev holds rays.nx*rays.ny records in ray order
 * (j*nx + i):
 *   FP32 variants: float4 {x_hi, y_hi, x_lo, y_lo}; beta_x = x_hi + x_lo
 *                  exactly as a real number (x_lo = 0 for MLENS_PREC_FP32_NAIVE),
 *                  and the pixel is the exact floor of that real number
 *                  (to about 1e-14 relative) -- the float32 rule spelled out in
 *                  the library's documentation of its binning step;
 *   MLENS_PREC_FP64: double2 {x, y}.
 * beta_dev must be 16-byte aligned and hold 16 * nx * ny bytes.
 */
int mlens_shoot_beta(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                     void *beta_dev, uint32_t flags, mlens_stats *stats_host, void *stream);

/*
 * mlens_shoot_rows -- mlens_shoot (or mlens_shoot_beta) restricted to the ray
 * rows [row_begin, row_end) of the grid `rays`.  Section 2.2 runs the method
 * with several MPI tasks, each tracing part of the rays into its own map, and
 * reduces the maps into one; this is one task's part.  Rays keep their
 * positions in the whole grid, and the launch shape, the star split (chosen for
 * the whole grid) and therefore every ray's beta are those of the whole-grid
 * call, so the maps of bands that cover the grid add up to the whole map bit for
 * bit (uint32 addition; a sum reduction across processes is exact).
 *   row_begin, row_end  0 <= row_begin <= row_end <= rays.ny, each a multiple
 *              of MLENS_ROW_ALIGN or row_end = rays.ny; 0, 0 = all rows.
 *   beta_dev   nullable; as for mlens_shoot_beta (the whole grid's
 *              rays.nx*rays.ny records), only the band's records are written.
 *   counts_dev, flags, stats_host, stream  as for mlens_shoot; stats count the
 *              band's rays (rays_total = rays.nx * (row_end - row_begin)).
 * Errors: MLENS_ERR_ARG (rows not aligned or out of range, and as mlens_shoot),
 * MLENS_ERR_CUDA.
 */
#define MLENS_ROW_ALIGN 32
int mlens_shoot_rows(mlens_ctx *ctx, const mlens_grid *rays, int32_t row_begin, int32_t row_end,
                     const mlens_grid *src, uint32_t *counts_dev, void *beta_dev, uint32_t flags,
                     mlens_stats *stats_host, void *stream);

/*
 * mlens_trace -- FP64 deflection at arbitrary image positions (Eq. 2-3), for
 * verification and for generating exact targets.  Uses the IEEE FP64 kernel
 * whatever the context's precision.
 *   theta_host k x 2 positions; beta_host receives k x 2 source positions.
 * Synchronous (copies in, runs on `stream`, waits, copies out).  Allocates and
 * frees a device buffer of 32*k bytes.
 */
int mlens_trace(mlens_ctx *ctx, const double *theta_host, int64_t k, double *beta_host, void *stream);

/*
 * mlens_bin -- the binning step of Algorithm 1 alone: count float-pair source
 * positions (the records mlens_shoot_beta writes for the FP32 variants) into a
 * source map with the same exact rule and the same privatised histogram.
 *   beta_dev   n float4 records {x_hi, y_hi, x_lo, y_lo}, device, 16-byte aligned.
 *   n          number of records, 0 <= n < 2^40.
 *   counts_dev as for mlens_shoot.
 * Needs no context: the scratch counters live in a per-device buffer the
 * library allocates on first use.
 */
int mlens_bin(const void *beta_dev, int64_t n, const mlens_grid *src, uint32_t *counts_dev, uint32_t flags,
              mlens_stats *stats_host, void *stream);

/*
 * mlens_bin_grid -- mlens_bin for records that form a ray grid: beta_dev holds
 * rays->nx * rays->ny records in the row-major order mlens_shoot_beta writes
 * (record j * nx + i is ray (i, j); only nx and ny of `rays` are used, and they
 * are checked like a shooting grid's).  The map is the same as mlens_bin's on
 * the same records; the kernel bins 64 x 64 blocks of neighbouring rays per CTA,
 * which keeps most increments in its shared-memory window.  Stats count all
 * nx * ny records.
 */
int mlens_bin_grid(const void *beta_dev, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                   uint32_t flags, mlens_stats *stats_host, void *stream);

/* Source intensity profiles of mlens_convolve. */
#define MLENS_PROFILE_GAUSSIAN 0
#define MLENS_PROFILE_DISK 1

/*
 * mlens_convolve -- the map convolved with a background source's intensity
 * profile.  Section 1: given a model of the source's size and intensity
 * profile, the magnification pattern yields simulated light curves; the
 * convolved map is the source's total magnification at each source position.
 *   out[j][i] = scale * sum_{(di,dj) in K} w(di,dj) * counts[j+dj][i+di]
 * with counts = 0 outside the map and the weights normalised to sum 1 over
 * their support K.  Offsets are measured in theta_E with the map's pixel widths
 * dx = (x1-x0)/nx, dy = (y1-y0)/ny (pixels need not be square).
 *   profile MLENS_PROFILE_GAUSSIAN: w proportional to exp(-|d|^2 / (2 size^2)),
 *              |di| <= ceil(4 size/dx), |dj| <= ceil(4 size/dy); the normalised
 *              1-D weights multiply.  FP32 arithmetic (two separable passes);
 *              needs 0 < size and 4 size <= 256 pixels along both axes.
 *   profile MLENS_PROFILE_DISK: a uniform disk of radius size (>= 0; 0 = the
 *              map itself): K = {(di dx)^2 + (dj dy)^2 <= size^2}, w = 1/|K|.
 *              Sums are exact integers; out = (float)(sum * (scale / |K|)) in
 *              FP64.  At most 4096 pixel rows in the support.
 *   counts_dev src->ny x src->nx uint32 counts (as mlens_shoot writes), device,
 *              4-byte aligned; pixel values above 2^24 lose precision in the
 *              Gaussian's FP32 passes.
 *   scale      multiplies the result: 1 = weighted counts; the value of
 *              mlens_magnification_scale turns counts into magnification.
 *   out_dev    src->ny x src->nx float32, device, 4-byte aligned, not
 *              overlapping counts_dev.
 *   work_dev   NULL, or caller-owned device workspace of at least
 *              mlens_convolve_workspace bytes (work_bytes), 256-byte aligned,
 *              overlapping neither map.  With a workspace the call allocates
 *              nothing and is asynchronous on `stream` (it can be captured in a
 *              CUDA graph); with NULL the library allocates the workspace (4
 *              bytes per pixel for the Gaussian, 8 for the disk), frees it
 *              before returning, and so synchronises `stream`.
 * The weights / half-widths are computed on the device from the definition
 * above (FP64, no contraction).  Errors: MLENS_ERR_ARG, MLENS_ERR_NOMEM,
 * MLENS_ERR_CUDA.
 */
int mlens_convolve(const uint32_t *counts_dev, const mlens_grid *src, int32_t profile, double size, double scale,
                   float *out_dev, void *work_dev, uint64_t work_bytes, void *stream);

/*
 * mlens_convolve_workspace -- bytes of device workspace mlens_convolve needs for
 * this map, profile and size (the normalised weights or the support's row
 * half-widths, and one map-sized buffer).  Host arithmetic only.
 * Errors: MLENS_ERR_ARG (as mlens_convolve's checks of src, profile and size).
 */
int mlens_convolve_workspace(const mlens_grid *src, int32_t profile, double size, uint64_t *bytes_out);

/*
 * mlens_light_curve -- a (convolved) map sampled along a straight source track:
 * npts points evenly spaced from (bx0, by0) to (bx1, by1) in theta_E (the
 * first point when npts = 1), each the bilinear interpolation between the
 * pixel centres (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy) around it, constant
 * beyond the outermost centres.  FP64 arithmetic, float32 output; asynchronous
 * on `stream`.
 *   map_dev    src->ny x src->nx float32 (e.g. mlens_convolve's output), device.
 *   out_dev    npts float32, device.
 * Errors: MLENS_ERR_ARG (npts < 1, non-finite end points, bad map grid),
 * MLENS_ERR_CUDA.
 */
int mlens_light_curve(const float *map_dev, const mlens_grid *src, double bx0, double by0, double bx1, double by1,
                      int32_t npts, float *out_dev, void *stream);

/*
 * mlens_magnification_scale -- A_lens / (N_rays * A_pix) for a ray grid and a
 * source map: a pixel receiving its mean share of rays (magnification 1) holds
 * N_rays * A_pix / A_lens of them, so magnification = counts * scale.
 * Host arithmetic only.  Errors: MLENS_ERR_ARG.
 */
int mlens_magnification_scale(const mlens_grid *rays, const mlens_grid *src, double *scale_out);

/*
 * mlens_shoot_noalloc -- mlens_shoot for callers that must not allocate device
 * memory: plugins whose host application owns every device allocation (its own
 * pool, its own accounting), and real-time loops that may not enter the CUDA
 * allocator (cudaMalloc and cudaFree can synchronise the device and take an
 * unbounded time).  It takes no context: the caller passes the stars already on
 * the device, and the only working memory is a fixed array compiled into the
 * library.
 * The paper has no counterpart; it is a deployment variant of the same FP32
 * kernel (MLENS_PREC_FP32, 8 rays per thread, 256-star stages, fma_pairs = 1, no
 * star split: a context's default tuning), so it produces the same map as
 * mlens_create + mlens_shoot (split 1) on the same float32 stars.
 *   stars_dev  n records float4 {x, y, m, unused} on the current device,
 *              16-byte aligned, caller-owned.  The values are not checked:
 *              non-finite entries give non-finite beta for the rays they touch.
 *   n          0 <= n <= MLENS_NOALLOC_MAX_STARS.
 *   kappa_c, gamma1, gamma2, rays, src, counts_dev, flags, stream
 *              as for mlens_create / mlens_shoot.
 *   stats_host nullable; when given, the call copies the counters back and
 *              waits for `stream` before it returns (as mlens_shoot does).
 * Working memory: one file-scope device array of MLENS_NOALLOC_MAX_STARS + 32
 * star records plus four 64-bit counters (three used; about 1 MiB), held on
 * every device that loads the library until the process exits.  Each call copies
 * the stars into it (padding the tail) and clears the counters on `stream` before
 * the kernel runs; the array keeps the last call's contents afterwards.  All
 * calls share that one array, so calls whose GPU work overlaps (different
 * streams, or different host threads) race and corrupt each other's maps:
 * serialise them.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture begins.  The
 * address is not looked up again after cudaDeviceReset, so calls after a reset
 * of the device in the same process are not supported.
 * Errors: MLENS_ERR_ARG (n above the maximum, bad grid, NULL or misaligned
 * pointer, non-finite lens terms), MLENS_ERR_CUDA.
 */
#define MLENS_NOALLOC_MAX_STARS 65536
int mlens_shoot_noalloc(const void *stars_dev, int64_t n, double kappa_c, double gamma1, double gamma2,
                        const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev, uint32_t flags,
                        mlens_stats *stats_host, void *stream);

/* ------------------------------------------------------------- batching */
/*
 * Many independent fields in one launch.  Section 2.2 runs grids of independent
 * simulations over (<M*>, gamma, kappa_*, kappa_c), each its own map; a batch
 * shoots them all in one persistent kernel that pulls (field, ray tile) items
 * from a device work queue, heaviest fields first, captured once into a CUDA
 * graph and replayed.  Every field uses MLENS_PREC_FP32 whatever its context's
 * setting.  With the same launch shape (see mlens_set_tuning) a field's map is
 * identical to mlens_shoot's on its own.
 */
typedef struct mlens_batch mlens_batch;

/*
 * mlens_batch_create -- describe a batch.
 *   ctxs[nfields]        contexts created on the current device (1 <= nfields <= 2^20);
 *   rays[nfields], srcs[nfields]  per-field ray grid and source map (limits as mlens_shoot);
 *   counts_dev[nfields]  per-field maps (srcs[f].ny x srcs[f].nx uint32, device, caller-owned);
 *   flags                0 or MLENS_ACCUMULATE.
 * Contexts and maps must stay alive, and unchanged in size, while the batch exists.
 * Allocates about 300 bytes per field of device tables and one private stream.
 * Launch shape starts at 8 rays per thread, 256-star stages and fma_pairs = 1.
 */
int mlens_batch_create(mlens_batch **out, mlens_ctx *const *ctxs, int32_t nfields, const mlens_grid *rays,
                       const mlens_grid *srcs, uint32_t *const *counts_dev, uint32_t flags);

/* Set the launch shape (as mlens_set_tuning).  Waits for the device; the graph is
 * captured again at the next run. */
int mlens_batch_set_tuning(mlens_batch *b, int32_t rays_per_thread, int32_t star_stage, int32_t fma_pairs);

/*
 * mlens_batch_tune -- the autotuner: time the launch shapes (rays per thread 8
 * or 4, star stage 256 or 512, fma_pairs 0 or 1) on this batch (a warm-up and
 * two timed replays each, CUDA events on `stream`), keep the fastest and report
 * it (any output pointer may be NULL; *best_ms = -1 when the shape came from the
 * cache).  Results are cached per process by device and workload
 * signature (field count, ray grid, star counts bucketed by powers of two), and
 * appended to / read from the text file named by the environment variable
 * MLENS_TUNE_CACHE when it is set.  The maps are overwritten by the trial runs.
 */
int mlens_batch_tune(mlens_batch *b, void *stream, int32_t *rays_per_thread, int32_t *star_stage, int32_t *fma_pairs,
                     double *best_ms);

/*
 * mlens_batch_run -- shoot every field (graph launch on `stream`; the first run of a
 * launch shape captures the graph).  stats_host, if non-NULL, receives nfields
 * records and makes the call wait for the stream.
 */
int mlens_batch_run(mlens_batch *b, mlens_stats *stats_host, void *stream);

/* Free a batch (waits for its device).  NULL is ignored. */
void mlens_batch_destroy(mlens_batch *b);

/* One-shot batch: create, run once, wait for the stream, destroy. */
int mlens_shoot_batch(mlens_ctx *const *ctxs, int32_t nfields, const mlens_grid *rays, const mlens_grid *srcs,
                      uint32_t *const *counts_dev, uint32_t flags, mlens_stats *stats_host, void *stream);

/* ------------------------------------------------- learned far field */
/*
 * The direct sum costs N_rays x N_* (Section 1: the summation over the stars is
 * the CPU-intensive part); with 10^6 stars most of it is the smooth pull of
 * distant stars.  The learned-far-field variant splits the lens plane into
 * square cells aligned with the ray tiles.  For a ray in cell c the stars of
 * the 3 x 3 block of cells around c are summed exactly (FP32, re-centred,
 * Kahan); the other stars act through the cell's far field F(z) =
 * sum_far m_k / (z - z_k) (alpha_far = conj F), holomorphic on the block and
 * written as a series in v = (z - z_c)/s (s = half the cell diagonal) whose
 * coefficients are FP64 direct sums over the far stars.  Orders 0..order are
 * evaluated exactly; the remainder up to target_order, v^(order+1) q(v), is
 * learned through q (which enters the series as its next coefficient) by a
 * small neural field -- a 32-number latent code per cell and one shared MLP
 * 34 -> 64 -> 64 -> 2 (SiLU) -- trained on the GPU with BF16 tensor-core
 * kernels (FP32 accumulation) on samples of that remainder.  Every cell whose
 * held-out validation error exceeds `tolerance` falls back to the exact
 * direct sum over all stars, which reproduces mlens_shoot's result for its
 * rays bit for bit.  With use_network = 0 the series alone is used (ablation).
 */
typedef struct {
    int32_t cells_x;              /* cells across the ray box in x; rays.nx must be a multiple of 64*cells_x */
    int32_t order;                /* series order evaluated exactly, 0..16 (default 10) */
    int32_t target_order;         /* order of the far-field expansion the network learns up to, order < . <= 24 (24) */
    int32_t use_network;          /* 1: learn the remainder (default); 0: series only */
    int64_t train_samples;        /* distinct training samples (2^24) */
    int32_t epochs;               /* passes over them (48) */
    int32_t batch;                /* samples per optimiser step, >= 128 (77824) */
    float lr_weights, lr_latents; /* Adam learning rates, cosine-decayed to 5 % (3.9e-3, 6.5e-2) */
    int32_t val_samples_per_cell; /* held-out samples per cell for validation (64) */
    double tolerance;             /* max validation error allowed per cell, theta_E (1e-6) */
    uint64_t seed;                /* seed of the counter-based sample and weight generators */
} mlens_fit_params;

typedef struct {
    int32_t cells, cells_fallback;     /* ray cells, and those falling back to the exact sum */
    int64_t tiles, tiles_fallback;     /* 64 x 32-ray tiles, and those on fallback cells */
    int64_t train_steps;
    double final_loss;                 /* mean squared error of the last step (cell-normalised units) */
    double val_max_err_net, val_mean_err_net;       /* |alpha_far error| with the network (theta_E; -1 if unused) */
    double val_max_err_series, val_mean_err_series; /* the same without the network (series to `order` only) */
    double seconds_coefficients, seconds_train, seconds_validate;
} mlens_fit_report;

typedef struct {
    int32_t cells_x, cells_y;       /* ray cells */
    double grid_x0, grid_y0, cell_width;  /* cell grid incl. a one-cell ring: cell (ix, iy) covers
                                             [x0 + ix w, x0 + (ix+1) w) x [y0 + iy w, ...) */
    int32_t grid_nx, grid_ny;       /* = cells_x + 2, cells_y + 2; ray cell (cx, cy) is grid cell (cx+1, cy+1) */
    int32_t order, target_order, use_network;
    int32_t n_params, latent_dim;   /* network parameter count (flat FP32 layout), latent size */
    mlens_fit_report report;
} mlens_far_field_info;

/* Fill *p with the defaults listed above. */
void mlens_fit_params_default(mlens_fit_params *p);

/*
 * mlens_fit_far_field -- build the learned far field of ctx's stars for the ray
 * grid `rays` (params NULL = defaults): cell CSR of the stars, FP64 expansion
 * coefficients, network training (if enabled), validation, fallback flags and
 * the work list (fallback tiles first).  Synchronous on `stream`; allocates the
 * far-field state in the context (replacing any previous one).
 * Errors: MLENS_ERR_ARG (grid not divisible into square tile-aligned cells, bad
 * settings), MLENS_ERR_STATE (wrong device), MLENS_ERR_NOMEM, MLENS_ERR_CUDA.
 */
int mlens_fit_far_field(mlens_ctx *ctx, const mlens_grid *rays, const mlens_fit_params *params,
                        mlens_fit_report *report, void *stream);

/*
 * mlens_shoot_learned -- mlens_shoot with the fitted far field over the tiles of
 * `rays` (which must be the grid of the fit).  Near stars exact, far field from
 * the series and the network, flagged cells exact: their tiles run first as the
 * plain sum split over clusters of 8, 4 or 2 CTAs (the largest leaving 2048 stars
 * per slice; none below 4096 stars), so they equal
 * mlens_shoot with that mlens_set_star_split bit for bit; then one persistent
 * launch takes the learned tiles.
 * beta_dev as for mlens_shoot_beta (NULL to skip); other arguments as mlens_shoot.
 * row_begin/row_end restrict the call to ray rows [row_begin, row_end) (both
 * multiples of 32; 0, 0 = all rows); a restricted call copies a filtered work
 * list into a device buffer the context allocates on first use.
 * The network's tensor-core waits are bounded: if one gives up (not expected on a
 * working device) the kernel stops using the tensor cores, drains and frees its
 * tensor memory, and a call with stats_host returns MLENS_ERR_CUDA (the map is
 * invalid); a call without stats_host does not check.
 */
int mlens_shoot_learned(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                        void *beta_dev, int32_t row_begin, int32_t row_end, uint32_t flags, mlens_stats *stats_host,
                        void *stream);

/* Layout and fit report of the context's far field. */
int mlens_far_field_get_info(mlens_ctx *ctx, mlens_far_field_info *out);

/*
 * mlens_far_field_export -- copy far-field state to host arrays (each may be NULL):
 * params (n_params FP32), latents (cells x 32), flags (cells), coef (cells x
 * (target_order+1) x {re, im} FP64 series coefficients in v), cell_start
 * (grid_nx*grid_ny + 1 CSR offsets), per-cell validation maxima with and without
 * the network (FP32, theta_E).  Waits for the device.
 */
int mlens_far_field_export(mlens_ctx *ctx, float *params, float *latents, int32_t *flags, double *coef,
                           int32_t *cell_start, float *val_max_net, float *val_max_series);

/* Save the fitted network, latents and flags (not the stars) to a file; loading
 * it into a context with the same stars rebuilds the geometry and skips training. */
int mlens_save_far_field(mlens_ctx *ctx, const char *path);
int mlens_load_far_field(mlens_ctx *ctx, const char *path, void *stream);

/*
 * mlens_ff_eval -- the network kernel on explicit inputs, for verification:
 * params_dev (n_params FP32), z_dev (n x 32), u_dev (n x 2), t_dev (n x 2 targets,
 * may be NULL without gradients); outputs y_dev (n x 2, nullable), grads_dev
 * (n_params, gradient of mean |y - t|^2, nullable), dz_dev (n x 32 latent
 * gradients, nullable), *loss_host.  Synchronous; allocates 17 KB of scratch.
 */
int mlens_ff_eval(const float *params_dev, const float *z_dev, const float *u_dev, const float *t_dev, int64_t n,
                  float *y_dev, float *grads_dev, float *dz_dev, float *loss_host, void *stream);

/*
 * mlens_debug_wait_probe -- test aid for the failure path of the tensor-core waits
 * (training, validation, mlens_ff_eval, the learned shoot).  While on (nonzero),
 * each such launch's first completion wait polls an mbarrier nothing arrives on,
 * 1024 times, so the bounded wait runs out: the kernel flags it, drains its
 * in-flight tensor-core work (bounded), frees its tensor memory and returns, and
 * the call reports MLENS_ERR_CUDA (the learned shoot when stats_host is given).
 * No fault, no hang; contexts stay usable.  Process-wide; 0 turns it off.
 */
int mlens_debug_wait_probe(int32_t on);

/* Free a context's device memory (waits for its device).  NULL is ignored. */
void mlens_destroy(mlens_ctx *ctx);

/*
 * mlens_set_device_memory_limit -- a budget (bytes; 0 = none, the default) for the
 * device memory the library itself allocates (star copies, counters, batch and
 * far-field tables; never the caller's maps).  An allocation that would exceed it
 * fails with MLENS_ERR_NOMEM as if the device were full, leaving every existing
 * context usable.  The environment variable MLENS_DEVICE_MEMORY_LIMIT sets the
 * initial budget.  mlens_device_memory_in_use reports the bytes currently held.
 */
int mlens_set_device_memory_limit(uint64_t bytes);
uint64_t mlens_device_memory_in_use(void);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *mlens_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int mlens_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLENS_H */
