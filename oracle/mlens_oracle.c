/*
 * mlens_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * backward ray-shooting method of Chen et al., "Accelerating gravitational
 * microlensing simulations using the Xeon Phi coprocessor" (arXiv:1703.09707).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; it is compiled into its own shared object and used by the tests, by
 * the bench's CPU-baseline leg and by the smoke check.  It shares no code,
 * header, constant or helper with the CUDA library.
 *
 * What it computes (all in IEEE double, stars visited in input order):
 *   Eq. (3):  alpha(theta) = [[kc+g1, g2], [g2, kc-g1]] theta
 *                            + sum_k m_k (theta - theta_k) / |theta - theta_k|^2
 *   Eq. (2):  beta = theta - alpha
 *   Algorithm 1: for every ray of a uniform lens-plane grid evaluate theta,
 *             alpha, beta, convert beta to source-pixel coordinates and, when
 *             the pixel is inside the source window, add one to mag[j_s][i_s].
 *
 * Readings of points the paper leaves open (listed with the others in the
 * design notes):
 *   - rays sit at cell centres: theta_x(i) = x0 + (i + 1/2) (x1 - x0) / nx;
 *   - pixel conversion is floor((beta_x - x0) * (nx / (x1 - x0))), lower edge
 *     inclusive, upper edge exclusive; the same for y;
 *   - a ray with a non-finite beta (a ray exactly on a star gives 0/0) is not
 *     binned and is counted as "nan"; a finite beta outside the window is
 *     counted as "out";
 *   - the map is row-major, row = y pixel (mag[j_s, i_s] in Algorithm 1).
 *
 * orc_rebin_pair() is different in kind: it is the float32 binning rule the
 * GPU kernels are specified to follow (a float-pair beta converted to a pixel
 * with a fixed sequence of IEEE float32 operations), written out again here
 * so that a GPU map can be re-binned on the CPU from the GPU's own beta and
 * compared bit for bit.  Build with -ffp-contract=off so that the compiler
 * adds no fused multiply-adds of its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double x0, x1, y0, y1;
    int32_t nx, ny;
} orc_grid;

/* ---------------------------------------------------------------- Eq. (3) */

/* Deflection of one ray: smooth + shear term alpha_0 (first term of Eq. 3)
 * plus the direct sum over all stars (second term). */
static void alpha_one(double tx, double ty, const double *xy, const double *m, int64_t n,
                      double kc, double g1, double g2, double *ax, double *ay)
{
    double sx = (kc + g1) * tx + g2 * ty;
    double sy = g2 * tx + (kc - g1) * ty;
    for (int64_t k = 0; k < n; ++k) {
        double dx = tx - xy[2 * k];
        double dy = ty - xy[2 * k + 1];
        double r2 = dx * dx + dy * dy;
        sx += m[k] * dx / r2;
        sy += m[k] * dy / r2;
    }
    *ax = sx;
    *ay = sy;
}

/* alpha for k arbitrary image positions theta (k x 2). */
void orc_alpha(const double *theta, int64_t k, const double *xy, const double *m, int64_t n,
               double kc, double g1, double g2, double *alpha, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < k; ++r)
        alpha_one(theta[2 * r], theta[2 * r + 1], xy, m, n, kc, g1, g2, &alpha[2 * r], &alpha[2 * r + 1]);
}

/* Scale of the terms of Eq. (3) at theta: |alpha_0| + sum_k m_k / |theta - theta_k|.
 * Any floating-point evaluation of the sum has an absolute error proportional to
 * this, so |alpha_computed - alpha| / scale is the error measure that stays
 * meaningful where alpha itself nearly cancels. */
void orc_alpha_scale(const double *theta, int64_t k, const double *xy, const double *m, int64_t n,
                     double kc, double g1, double g2, double *scale, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < k; ++r) {
        double tx = theta[2 * r], ty = theta[2 * r + 1];
        double sx = (kc + g1) * tx + g2 * ty;
        double sy = g2 * tx + (kc - g1) * ty;
        double acc = sqrt(sx * sx + sy * sy);
        for (int64_t s = 0; s < n; ++s) {
            double dx = tx - xy[2 * s];
            double dy = ty - xy[2 * s + 1];
            acc += m[s] / sqrt(dx * dx + dy * dy);
        }
        scale[r] = acc;
    }
}

/* Jacobian d alpha / d theta of Eq. (3): M + sum_k m_k (r^2 I - 2 d d^T) / r^4,
 * d = theta - theta_k; out = {J11, J12, J22} per position (J is symmetric).
 * It bounds how far alpha moves when a position is rounded. */
void orc_alpha_jacobian(const double *theta, int64_t k, const double *xy, const double *m, int64_t n,
                        double kc, double g1, double g2, double *jac, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < k; ++r) {
        double tx = theta[2 * r], ty = theta[2 * r + 1];
        double j11 = kc + g1, j12 = g2, j22 = kc - g1;
        for (int64_t s = 0; s < n; ++s) {
            double dx = tx - xy[2 * s];
            double dy = ty - xy[2 * s + 1];
            double r2 = dx * dx + dy * dy;
            double w = m[s] / (r2 * r2);
            j11 += w * (dy * dy - dx * dx);
            j12 += w * (-2.0 * dx * dy);
            j22 += w * (dx * dx - dy * dy);
        }
        jac[3 * r] = j11;
        jac[3 * r + 1] = j12;
        jac[3 * r + 2] = j22;
    }
}

/* ------------------------------------------------ cells: near and far stars */
/* The learned-far-field variant splits the lens plane into a grid of square
 * cells; for a ray in cell c the "near" stars are those in the 3 x 3 block of
 * cells around c (clipped to the grid) and every other star (including stars
 * outside the grid) is "far".  Cell (ix, iy), 0 <= ix < nx, 0 <= iy < ny, covers
 * [x0 + ix w, x0 + (ix+1) w) x [y0 + iy w, y0 + (iy+1) w); index iy*nx + ix. */
typedef struct {
    double x0, y0, w;
    int32_t nx, ny;
} orc_cells;

static int64_t cell_index(double x, double y, const orc_cells *c)
{
    double fx = floor((x - c->x0) / c->w), fy = floor((y - c->y0) / c->w);
    if (!(fx >= 0.0 && fx < (double)c->nx && fy >= 0.0 && fy < (double)c->ny)) return -1;
    return (int64_t)fy * c->nx + (int64_t)fx;
}

void orc_cell_index(const double *xy, int64_t k, const orc_cells *c, int64_t *out)
{
    for (int64_t r = 0; r < k; ++r) out[r] = cell_index(xy[2 * r], xy[2 * r + 1], c);
}

static int is_near(int64_t star_cell, int64_t ray_cell, int32_t n)
{
    if (star_cell < 0 || ray_cell < 0) return 0;
    int64_t sx = star_cell % n, sy = star_cell / n, rx = ray_cell % n, ry = ray_cell / n;  /* n = cells per row */
    return (sx - rx <= 1 && rx - sx <= 1 && sy - ry <= 1 && ry - sy <= 1);
}

/* Star term of Eq. (3) at theta split by the cell rule: out_near and out_far
 * (either may be NULL), both k x 2.  ray_cell[r] is the cell the ray belongs to. */
void orc_split_alpha(const double *theta, const int64_t *ray_cell, int64_t k, const double *xy, const double *m,
                     int64_t n, const orc_cells *c, double *out_near, double *out_far, int nthreads)
{
    int64_t *scell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) scell[s] = cell_index(xy[2 * s], xy[2 * s + 1], c);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t r = 0; r < k; ++r) {
        double tx = theta[2 * r], ty = theta[2 * r + 1];
        double nx = 0.0, ny = 0.0, fx = 0.0, fy = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            double dx = tx - xy[2 * s];
            double dy = ty - xy[2 * s + 1];
            double r2 = dx * dx + dy * dy;
            double ax = m[s] * dx / r2, ay = m[s] * dy / r2;
            if (is_near(scell[s], ray_cell[r], c->nx)) {
                nx += ax;
                ny += ay;
            } else {
                fx += ax;
                fy += ay;
            }
        }
        if (out_near) {
            out_near[2 * r] = nx;
            out_near[2 * r + 1] = ny;
        }
        if (out_far) {
            out_far[2 * r] = fx;
            out_far[2 * r + 1] = fy;
        }
    }
    free(scell);
}

/* Local (Taylor) expansion of the far field of each listed cell about its
 * centre z_c.  With z = x + i y, the star term of Eq. (3) is the complex
 * conjugate of F(z) = sum_k m_k / (z - z_k), holomorphic away from the stars;
 * for the far stars of cell c,
 *     F(z) = sum_{p>=0} a_p (z - z_c)^p,   a_p = - sum_far m_k / (z_k - z_c)^(p+1).
 * out[(cell i, p)] = (Re a_p, Im a_p) scaled by s^p (s = scale): the coefficients
 * of the series in (z - z_c)/s.  FP64, stars in input order. */
void orc_local_coeffs(const int64_t *cells, int64_t ncell, int32_t P, double scale, const double *xy,
                      const double *m, int64_t n, const orc_cells *c, double *out, int nthreads)
{
    int64_t *scell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) scell[s] = cell_index(xy[2 * s], xy[2 * s + 1], c);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < ncell; ++i) {
        int64_t cc = cells[i];
        double zx = c->x0 + ((double)(cc % c->nx) + 0.5) * c->w;
        double zy = c->y0 + ((double)(cc / c->nx) + 0.5) * c->w;
        double *o = out + (size_t)i * 2 * (size_t)(P + 1);
        for (int32_t p = 0; p <= P; ++p) o[2 * p] = o[2 * p + 1] = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            if (is_near(scell[s], cc, c->nx)) continue;
            /* w = scale / (z_k - z_c); term_p = -m w^(p+1) / scale */
            double dx = xy[2 * s] - zx, dy = xy[2 * s + 1] - zy;
            double d2 = dx * dx + dy * dy;
            double wr = scale * dx / d2, wi = -scale * dy / d2;
            double tr = -m[s] * wr / scale, ti = -m[s] * wi / scale;
            for (int32_t p = 0; p <= P; ++p) {
                o[2 * p] += tr;
                o[2 * p + 1] += ti;
                double nr = tr * wr - ti * wi, ni = tr * wi + ti * wr;
                tr = nr;
                ti = ni;
            }
        }
    }
    free(scell);
}

/* ------------------------------------------------------ grid and binning */

static double ray_x(const orc_grid *g, int64_t i) { return g->x0 + ((double)i + 0.5) * ((g->x1 - g->x0) / g->nx); }
static double ray_y(const orc_grid *g, int64_t j) { return g->y0 + ((double)j + 0.5) * ((g->y1 - g->y0) / g->ny); }

/* Source-pixel conversion of Algorithm 1.  Returns the linear pixel index
 * j_s*nx + i_s, or -1 for a finite beta outside the window, or -2 for a
 * non-finite beta. */
static int64_t pixel_of(double bx, double by, const orc_grid *s)
{
    if (!isfinite(bx) || !isfinite(by)) return -2;
    double ux = floor((bx - s->x0) * ((double)s->nx / (s->x1 - s->x0)));
    double uy = floor((by - s->y0) * ((double)s->ny / (s->y1 - s->y0)));
    if (ux < 0.0 || ux >= (double)s->nx || uy < 0.0 || uy >= (double)s->ny) return -1;
    return (int64_t)uy * s->nx + (int64_t)ux;
}

void orc_pixels(const double *beta, int64_t k, const orc_grid *src, int64_t *pix)
{
    for (int64_t r = 0; r < k; ++r) pix[r] = pixel_of(beta[2 * r], beta[2 * r + 1], src);
}

void orc_ray_theta(const orc_grid *rays, const int64_t *idx, int64_t k, double *theta)
{
    for (int64_t r = 0; r < k; ++r) {
        int64_t i = idx[r] % rays->nx, j = idx[r] / rays->nx;
        theta[2 * r] = ray_x(rays, i);
        theta[2 * r + 1] = ray_y(rays, j);
    }
}

/* ---------------------------------------------------------- Algorithm 1 */

/* Full backward ray-shooting of one map.  counts (ny x nx) is overwritten.
 * stats = {rays_total, rays_binned, rays_out, rays_nan}. */
void orc_shoot(const orc_grid *rays, const orc_grid *src, const double *xy, const double *m, int64_t n,
               double kc, double g1, double g2, uint32_t *counts, uint64_t *stats, int nthreads)
{
    int64_t npix = (int64_t)src->nx * src->ny;
    memset(counts, 0, sizeof(uint32_t) * (size_t)npix);
    uint64_t binned = 0, out = 0, nan = 0;
    int64_t nrx = rays->nx, nry = rays->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for collapse(2) schedule(dynamic, 256) reduction(+ : binned, out, nan)
#endif
    for (int64_t j = 0; j < nry; ++j) {
        for (int64_t i = 0; i < nrx; ++i) {
            double tx = ray_x(rays, i), ty = ray_y(rays, j), ax, ay;
            alpha_one(tx, ty, xy, m, n, kc, g1, g2, &ax, &ay);
            double bx = tx - ax, by = ty - ay;
            int64_t p = pixel_of(bx, by, src);
            if (p >= 0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                counts[p] += 1u;
                binned++;
            } else if (p == -1) {
                out++;
            } else {
                nan++;
            }
        }
    }
    stats[0] = (uint64_t)(nrx * nry);
    stats[1] = binned;
    stats[2] = out;
    stats[3] = nan;
}

/* beta (k x 2) of selected rays of the grid, identified by linear index j*nx+i. */
void orc_beta_rays(const orc_grid *rays, const int64_t *idx, int64_t k, const double *xy, const double *m,
                   int64_t n, double kc, double g1, double g2, double *beta, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t r = 0; r < k; ++r) {
        int64_t i = idx[r] % rays->nx, j = idx[r] / rays->nx;
        double tx = ray_x(rays, i), ty = ray_y(rays, j), ax, ay;
        alpha_one(tx, ty, xy, m, n, kc, g1, g2, &ax, &ay);
        beta[2 * r] = tx - ax;
        beta[2 * r + 1] = ty - ay;
    }
}

/* ------------------------------------------- float-pair binning (GPU rule) */

/* Error-free sum of two floats (Knuth's TwoSum). */
static void two_sum_f(float a, float b, float *s, float *e)
{
    float x = a + b;
    float bb = x - a;
    float err = (a - (x - bb)) + (b - bb);
    *s = x;
    *e = err;
}

/* Pixel coordinate of one axis: u = (b_hi + b_lo - x0) * (n / (x1 - x0)),
 * evaluated as a float pair and floored exactly.  Returns -1 for out of
 * window (the caller has already rejected non-finite input). */
static int32_t pair_axis(float bh, float bl, double x0, double x1, int32_t n)
{
    double sd = (double)n / (x1 - x0);
    float x0h = (float)x0, x0l = (float)(x0 - (double)x0h);
    float sh = (float)sd, sl = (float)(sd - (double)sh);
    float dh, dl;
    two_sum_f(bh, -x0h, &dh, &dl);
    float t = bl - x0l;
    dl = dl + t;
    two_sum_f(dh, dl, &dh, &dl);
    float uh = dh * sh;
    float ul = fmaf(dh, sh, -uh);
    ul = fmaf(dh, sl, ul);
    ul = fmaf(dl, sh, ul);
    two_sum_f(uh, ul, &uh, &ul);
    if (!(uh == uh) || isinf(uh)) return -1;
    float p = floorf(uh);
    if (p == uh && ul < 0.0f) p = p - 1.0f;
    if (p < 0.0f || p >= (float)n) return -1;
    return (int32_t)p;
}

/* Re-bin a GPU beta buffer: beta4[r] = {x_hi, y_hi, x_lo, y_lo}.  counts are
 * overwritten.  stats = {total, binned, out, nan}.  Sequential on purpose. */
void orc_rebin_pair(const float *beta4, int64_t k, const orc_grid *src, uint32_t *counts, uint64_t *stats)
{
    memset(counts, 0, sizeof(uint32_t) * (size_t)src->nx * (size_t)src->ny);
    uint64_t binned = 0, out = 0, nan = 0;
    for (int64_t r = 0; r < k; ++r) {
        float xh = beta4[4 * r], yh = beta4[4 * r + 1], xl = beta4[4 * r + 2], yl = beta4[4 * r + 3];
        if (!isfinite(xh) || !isfinite(yh) || !isfinite(xl) || !isfinite(yl)) { nan++; continue; }
        int32_t px = pair_axis(xh, xl, src->x0, src->x1, src->nx);
        int32_t py = pair_axis(yh, yl, src->y0, src->y1, src->ny);
        if (px < 0 || py < 0) { out++; continue; }
        counts[(int64_t)py * src->nx + px] += 1u;
        binned++;
    }
    stats[0] = (uint64_t)k;
    stats[1] = binned;
    stats[2] = out;
    stats[3] = nan;
}

/* Pixel index of each float-pair beta under the GPU rule (-1 out, -2 nan). */
void orc_pair_pixels(const float *beta4, int64_t k, const orc_grid *src, int64_t *pix)
{
    for (int64_t r = 0; r < k; ++r) {
        float xh = beta4[4 * r], yh = beta4[4 * r + 1], xl = beta4[4 * r + 2], yl = beta4[4 * r + 3];
        if (!isfinite(xh) || !isfinite(yh) || !isfinite(xl) || !isfinite(yl)) { pix[r] = -2; continue; }
        int32_t px = pair_axis(xh, xl, src->x0, src->x1, src->nx);
        int32_t py = pair_axis(yh, yl, src->y0, src->y1, src->ny);
        pix[r] = (px < 0 || py < 0) ? -1 : (int64_t)py * src->nx + px;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
