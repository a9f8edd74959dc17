// api.cu -- the extern "C" boundary of libmlens (declared in include/mlens.h):
// argument checking, device buffers owned by a context, kernel selection and
// error reporting.  Every step of the computation runs in the kernels of the
// other translation units; nothing here computes on the host except the
// per-grid constants the kernels take by value.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "mlens_internal.h"

using namespace mlens;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    clear_pending_error();
    return e == cudaErrorMemoryAllocation ? MLENS_ERR_NOMEM : MLENS_ERR_CUDA;
}

#define MLENS_CUDA(call, what)                    \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool finite_box(const mlens_grid &g)
{
    return std::isfinite(g.x0) && std::isfinite(g.x1) && std::isfinite(g.y0) && std::isfinite(g.y1) &&
           g.x1 > g.x0 && g.y1 > g.y0;
}

int check_rays(const mlens_grid *g)
{
    if (!g) return fail(MLENS_ERR_ARG, "rays grid is NULL");
    if (!finite_box(*g)) return fail(MLENS_ERR_ARG, "rays grid box must be finite with x1 > x0 and y1 > y0");
    if (g->nx < 1 || g->ny < 1 || g->nx > (1 << 20) || g->ny > (1 << 20))
        return fail(MLENS_ERR_ARG, "rays grid needs 1 <= nx, ny <= 2^20");
    return MLENS_OK;
}

int check_src(const mlens_grid *g)
{
    if (!g) return fail(MLENS_ERR_ARG, "source grid is NULL");
    if (!finite_box(*g)) return fail(MLENS_ERR_ARG, "source box must be finite with x1 > x0 and y1 > y0");
    if (g->nx < 1 || g->ny < 1 || (int64_t)g->nx * g->ny > (int64_t(1) << 30))
        return fail(MLENS_ERR_ARG, "source map needs nx, ny >= 1 and nx*ny <= 2^30");
    return MLENS_OK;
}

int check_current_device(int want)
{
    int dev = -1;
    MLENS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (want >= 0 && dev != want)
        return fail(MLENS_ERR_STATE, "the context belongs to another CUDA device than the current one");
    return MLENS_OK;
}

// per-device scratch counters for calls made without a context (mlens_bin)
std::mutex g_scratch_mu;
std::vector<unsigned long long *> g_scratch;

int device_scratch(unsigned long long **out)
{
    int dev = -1;
    MLENS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if ((int)g_scratch.size() <= dev) g_scratch.resize(dev + 1, nullptr);
    if (!g_scratch[dev]) MLENS_CUDA(dmalloc(&g_scratch[dev], 4 * sizeof(unsigned long long)), "cudaMalloc(scratch)");
    *out = g_scratch[dev];
    return MLENS_OK;
}

AxisPair make_axis(double x0, double x1, int n)
{
    AxisPair a;
    const double s = (double)n / (x1 - x0);
    a.x0h = (float)x0;
    a.x0l = (float)(x0 - (double)a.x0h);
    a.sh = (float)s;
    a.sl = (float)(s - (double)a.sh);
    a.sh2 = 2.0f * std::fabs(a.sh);
    const double tq = 2.0 * std::fabs((double)a.x0l) * std::fabs((double)a.sh) + 0x1p-100;
    a.tq = (float)tq;
    if ((double)a.tq < tq) a.tq = std::nextafter(a.tq, INFINITY);
    a.n = n;
    return a;
}

int read_stats(unsigned long long *d_stats, uint64_t total, mlens_stats *st, cudaStream_t s)
{
    unsigned long long h[3];
    MLENS_CUDA(cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(stats)");
    MLENS_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    st->rays_total = total;
    st->rays_binned = h[0];
    st->rays_out = h[1];
    st->rays_nan = h[2];
    return MLENS_OK;
}

// Ray rows per tile of the FP32 kernels (the FP64 kernel's 4-row blocks divide it).
int tile_rows_of(const mlens_ctx *ctx) { return 8 * ctx->pairs_per_thread; }

// The global split's partials per pass (tile rows are taken in passes that fit).
constexpr size_t kGsplitBytes = size_t(256) << 20;

// CTAs per tile for the FP32 re-centred kernel: the split star sum runs with the
// default stage (and either reciprocal split).
int effective_split(const mlens_ctx *ctx, const RayGrid &r)
{
    if (ctx->precision != MLENS_PREC_FP32 || ctx->star_stage != kSplitStage) return 1;
    if (ctx->star_split) return ctx->star_split;
    return auto_star_split(r, ctx->pairs_per_thread, ctx->n_pad, ctx->nsm);
}

// Rays rows [row0, row1) of the grid (row1 < 0: all rows).
int shoot_impl(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts, void *beta,
               uint32_t flags, mlens_stats *stats, void *stream, int row0 = 0, int row1 = -1)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    int rc;
    if ((rc = check_rays(rays)) || (rc = check_src(src))) return rc;
    if (row1 < 0) row1 = rays->ny;
    if (row0 < 0 || row0 > row1 || row1 > rays->ny || row0 % MLENS_ROW_ALIGN != 0 ||
        (row1 % MLENS_ROW_ALIGN != 0 && row1 != rays->ny))
        return fail(MLENS_ERR_ARG, "rows must satisfy 0 <= row_begin <= row_end <= rays.ny, both multiples of "
                                   "MLENS_ROW_ALIGN (32) or row_end = rays.ny");
    if (!counts) return fail(MLENS_ERR_ARG, "counts_dev is NULL");
    if (((uintptr_t)counts & 3u) != 0) return fail(MLENS_ERR_ARG, "counts_dev must be 4-byte aligned");
    if (beta && ((uintptr_t)beta & 15u) != 0) return fail(MLENS_ERR_ARG, "beta_dev must be 16-byte aligned");
    if (flags & ~MLENS_ACCUMULATE) return fail(MLENS_ERR_ARG, "unknown flag bits");
    if ((rc = check_current_device(ctx->device))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)src->nx * (size_t)src->ny;
    if (!(flags & MLENS_ACCUMULATE))
        MLENS_CUDA(cudaMemsetAsync(counts, 0, npix * sizeof(uint32_t), s), "cudaMemsetAsync(counts)");
    MLENS_CUDA(cudaMemsetAsync(ctx->d_stats, 0, 3 * sizeof(unsigned long long), s), "cudaMemsetAsync(stats)");
    ShootArgs a{};
    a.stars = ctx->d_stars;
    a.nstars = ctx->n_pad;
    a.rays = make_ray_grid(*rays);
    a.bin = make_bin_grid(*src);
    a.lens = ctx->lens;
    a.counts = counts;
    a.stats = ctx->d_stats;
    a.beta_out = beta;
    cudaError_t e = cudaSuccess;
    // the split follows the whole grid, so a band of rows equals those rows of the
    // whole map bit for bit
    const int split = effective_split(ctx, a.rays);
    const int th = tile_rows_of(ctx);  // divides MLENS_ROW_ALIGN
    if (row1 > row0) {
        const int ty0 = row0 / th, ty1 = (row1 + th - 1) / th;
        if (ctx->precision == MLENS_PREC_FP64) {
            e = launch_shoot_fp64(a, s, row0, row1);
        } else if (split > kMaxClusterSplit) {
            // partials of up to kGsplitBytes per pass (at least one tile row), in a
            // context workspace grown on demand
            const int rpp = std::min(gsplit_rows_per_pass(a.rays, ctx->pairs_per_thread, split, kGsplitBytes),
                                     ty1 - ty0);
            const size_t need = gsplit_part_bytes(a.rays, ctx->pairs_per_thread, split, rpp);
            if (ctx->gpart_bytes < need) {
                if (ctx->d_gpart) dfree(ctx->d_gpart);
                ctx->d_gpart = nullptr;
                ctx->gpart_bytes = 0;
                MLENS_CUDA(dmalloc(&ctx->d_gpart, need), "cudaMalloc(split partials)");
                ctx->gpart_bytes = need;
            }
            e = launch_shoot_gsplit(a, ctx->pairs_per_thread, split, ctx->d_gpart, rpp, s, ty0, ty1, ctx->fma_pairs);
        } else if (split > 1) {
            e = launch_shoot_split(a, ctx->pairs_per_thread, split, s, ty0, ty1, ctx->fma_pairs);
        } else {
            e = launch_shoot_fp32(a, ctx->pairs_per_thread, ctx->precision == MLENS_PREC_FP32_NAIVE, s,
                                  ctx->star_stage, ctx->fma_pairs, ty0, ty1);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "shoot kernel launch");
    if (stats) return read_stats(ctx->d_stats, (uint64_t)rays->nx * (uint64_t)(row1 - row0), stats, s);
    return MLENS_OK;
}

}  // namespace

namespace mlens {

void set_last_error(const std::string &msg) { g_err = msg; }

namespace {
std::mutex g_mem_mu;
std::unordered_map<const void *, size_t> g_mem_sizes;
uint64_t g_mem_in_use = 0;
uint64_t g_mem_limit = 0;  // 0 = no budget
std::once_flag g_mem_env_once;

// The budget may also come from the environment (MLENS_DEVICE_MEMORY_LIMIT, bytes).
void read_env_limit()
{
    std::call_once(g_mem_env_once, [] {
        const char *v = getenv("MLENS_DEVICE_MEMORY_LIMIT");
        if (v) g_mem_limit = strtoull(v, nullptr, 10);
    });
}
}  // namespace

uint64_t mem_in_use()
{
    std::lock_guard<std::mutex> lk(g_mem_mu);
    return g_mem_in_use;
}

void set_mem_limit(uint64_t bytes)
{
    read_env_limit();
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_mem_limit = bytes;
}

cudaError_t dmalloc_raw(void **p, size_t bytes)
{
    read_env_limit();
    *p = nullptr;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (g_mem_limit && g_mem_in_use + bytes > g_mem_limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    g_mem_sizes[*p] = bytes;
    g_mem_in_use += bytes;
    return cudaSuccess;
}

void dfree(const void *p)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        auto it = g_mem_sizes.find(p);
        if (it != g_mem_sizes.end()) {
            g_mem_in_use -= it->second;
            g_mem_sizes.erase(it);
        }
    }
    cudaFree(const_cast<void *>(p));
}

BinGrid make_bin_grid(const mlens_grid &g)
{
    BinGrid b;
    b.ax = make_axis(g.x0, g.x1, g.nx);
    b.ay = make_axis(g.y0, g.y1, g.ny);
    b.x0 = g.x0;
    b.x1 = g.x1;
    b.y0 = g.y0;
    b.y1 = g.y1;
    b.nx = g.nx;
    b.ny = g.ny;
    return b;
}

// The value of the lowest set bit of x's significand (x = m 2^e, m odd: 2^e);
// +infinity for 0.
static double low_bit(double x)
{
    if (x == 0.0) return INFINITY;
    int e = 0;
    const double m = std::frexp(std::fabs(x), &e);  // m in [1/2, 1)
    const uint64_t M = (uint64_t)std::ldexp(m, 53);
    int tz = 0;
    while (((M >> tz) & 1u) == 0) ++tz;
    return std::ldexp(1.0, e - 53 + tz);
}

RayGrid make_ray_grid(const mlens_grid &g)
{
    RayGrid r;
    r.x0 = g.x0;
    r.x1 = g.x1;
    r.y0 = g.y0;
    r.y1 = g.y1;
    r.nx = g.nx;
    r.ny = g.ny;
    r.dx = (g.x1 - g.x0) / g.nx;
    r.dy = (g.y1 - g.y0) / g.ny;
    r.dxh = (float)r.dx;
    r.dxl = (float)(r.dx - (double)r.dxh);
    r.dyh = (float)r.dy;
    r.dyl = (float)(r.dy - (double)r.dyh);
    r.qx = std::ldexp(1.0, std::ilogb(r.dx));
    r.qy = std::ldexp(1.0, std::ilogb(r.dy));
    r.qxinv = 1.0 / r.qx;
    r.qyinv = 1.0 / r.qy;
    // Ray offsets from the tile centres are exact floats when every ray position
    // x0 + (i + 1/2) dx and every centre (0 or a multiple of qx) is a multiple of
    // one power of two g with all offsets below 2^24 g: g = the lowest set bit of
    // dx/2, x0 and qx; offsets stay within 6 tile extents.  Then the kernels need
    // no low parts (the workloads' dyadic grids); otherwise they add them.
    auto exact_axis = [](double x0, double d, double q, int tile) {
        const double g = std::min(std::min(low_bit(0.5 * d), low_bit(x0)), q);
        return 6.0 * tile * d < std::ldexp(g, 24);
    };
    r.lo = (exact_axis(g.x0, r.dx, r.qx, 64) && exact_axis(g.y0, r.dy, r.qy, 32)) ? 0 : 1;
    return r;
}

LensTerms make_lens_terms(double kc, double g1, double g2)
{
    LensTerms L;
    L.kc = kc;
    L.g1 = g1;
    L.g2 = g2;
    L.a11 = 1.0 - kc - g1;
    L.a12 = -g2;
    L.a22 = 1.0 - kc + g1;
    L.fa11 = (float)L.a11;
    L.fa12 = (float)L.a12;
    L.fa22 = (float)L.a22;
    L.fm11 = (float)(kc + g1);
    L.fm12 = (float)g2;
    L.fm22 = (float)(kc - g1);
    return L;
}

}  // namespace mlens

namespace {
int bin_impl(const void *beta_dev, int64_t n, int rnx, int rny, const mlens_grid *src, uint32_t *counts_dev,
             uint32_t flags, mlens_stats *stats_host, void *stream)
{
    int rc;
    if ((rc = check_src(src))) return rc;
    if (n > 0 && !beta_dev) return fail(MLENS_ERR_ARG, "beta_dev is NULL");
    if (!counts_dev) return fail(MLENS_ERR_ARG, "counts_dev is NULL");
    if (((uintptr_t)counts_dev & 3u) != 0) return fail(MLENS_ERR_ARG, "counts_dev must be 4-byte aligned");
    if (((uintptr_t)beta_dev & 15u) != 0) return fail(MLENS_ERR_ARG, "beta_dev must be 16-byte aligned");
    if (flags & ~MLENS_ACCUMULATE) return fail(MLENS_ERR_ARG, "unknown flag bits");
    unsigned long long *st = nullptr;
    if ((rc = device_scratch(&st))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)src->nx * (size_t)src->ny;
    if (!(flags & MLENS_ACCUMULATE))
        MLENS_CUDA(cudaMemsetAsync(counts_dev, 0, npix * sizeof(uint32_t), s), "cudaMemsetAsync(counts)");
    MLENS_CUDA(cudaMemsetAsync(st, 0, 3 * sizeof(unsigned long long), s), "cudaMemsetAsync(stats)");
    BinArgs a{};
    a.beta = reinterpret_cast<const float4 *>(beta_dev);
    a.n = n;
    a.rnx = rnx;
    a.rny = rny;
    a.bin = make_bin_grid(*src);
    a.counts = counts_dev;
    a.stats = st;
    cudaError_t e = launch_bin(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "bin kernel launch");
    if (stats_host) return read_stats(st, (uint64_t)n, stats_host, s);
    return MLENS_OK;
}
}  // namespace

extern "C" {

const char *mlens_last_error(void) { return g_err.c_str(); }

int mlens_set_device_memory_limit(uint64_t bytes)
{
    mlens::set_mem_limit(bytes);
    return MLENS_OK;
}

uint64_t mlens_device_memory_in_use(void) { return mlens::mem_in_use(); }

int mlens_version(void) { return 10000; }

int mlens_create(mlens_ctx **out, const double *xy, const double *m, int64_t n, double kappa_c, double gamma1,
                 double gamma2, int32_t precision)
{
    if (!out) return fail(MLENS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(MLENS_ERR_ARG, "n must satisfy 0 <= n < 2^31");
    if (n > 0 && (!xy || !m)) return fail(MLENS_ERR_ARG, "xy_host and m_host must be non-NULL when n > 0");
    if (!std::isfinite(kappa_c) || !std::isfinite(gamma1) || !std::isfinite(gamma2))
        return fail(MLENS_ERR_ARG, "kappa_c and gamma must be finite");
    if (precision < MLENS_PREC_FP32 || precision > MLENS_PREC_FP64)
        return fail(MLENS_ERR_ARG, "unknown precision");
    const int64_t n_pad = (n + kStarPad - 1) / kStarPad * kStarPad;
    std::vector<float4> h((size_t)n_pad, make_float4(kPadCoord, kPadCoord, 0.0f, 0.0f));
    for (int64_t k = 0; k < n; ++k) {
        const double x = xy[2 * k], y = xy[2 * k + 1], mk = m[k];
        if (!std::isfinite(x) || !std::isfinite(y) || std::fabs(x) >= 1e12 || std::fabs(y) >= 1e12)
            return fail(MLENS_ERR_ARG, "star " + std::to_string(k) + ": position must be finite with |x|,|y| < 1e12");
        if (!std::isfinite(mk) || mk < 0.0)
            return fail(MLENS_ERR_ARG, "star " + std::to_string(k) + ": mass must be finite and >= 0");
        h[(size_t)k] = make_float4((float)x, (float)y, (float)mk, 0.0f);
    }
    int dev = -1;
    MLENS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop;
    MLENS_CUDA(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
        return fail(MLENS_ERR_UNSUPPORTED, "libmlens is built for sm_103a (GB300); current device is sm_" +
                                               std::to_string(prop.major) + std::to_string(prop.minor));
    mlens_ctx *c = new mlens_ctx();
    c->device = dev;
    c->nsm = prop.multiProcessorCount;
    c->n = n;
    c->n_pad = n_pad;
    c->lens = make_lens_terms(kappa_c, gamma1, gamma2);
    c->precision = precision;
    cudaError_t e = cudaSuccess;
    if (n_pad > 0) e = dmalloc(&c->d_stars, (size_t)n_pad * sizeof(float4));
    if (e == cudaSuccess) e = dmalloc(&c->d_stats, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess && n_pad > 0)
        e = cudaMemcpy(c->d_stars, h.data(), (size_t)n_pad * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "mlens_create device setup");
        mlens_destroy(c);
        return rc;
    }
    *out = c;
    return MLENS_OK;
}

int mlens_set_precision(mlens_ctx *ctx, int32_t precision)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    if (precision < MLENS_PREC_FP32 || precision > MLENS_PREC_FP64) return fail(MLENS_ERR_ARG, "unknown precision");
    ctx->precision = precision;
    return MLENS_OK;
}

int mlens_set_tuning(mlens_ctx *ctx, int32_t rays_per_thread, int32_t star_stage, int32_t fma_pairs)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    if (rays_per_thread != 4 && rays_per_thread != 8) return fail(MLENS_ERR_ARG, "rays_per_thread must be 4 or 8");
    if (star_stage != 0 && star_stage != 128 && star_stage != 256 && star_stage != 512)
        return fail(MLENS_ERR_ARG, "star_stage must be 0 (default), 128, 256 or 512");
    if (fma_pairs != 0 && fma_pairs != 1) return fail(MLENS_ERR_ARG, "fma_pairs must be 0 or 1");
    ctx->pairs_per_thread = rays_per_thread / 2;
    ctx->star_stage = star_stage ? star_stage : 256;
    ctx->fma_pairs = fma_pairs;
    return MLENS_OK;
}

int mlens_set_star_split(mlens_ctx *ctx, int32_t split)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    if (split < 0 || split > kMaxSplit)
        return fail(MLENS_ERR_ARG, "split must be 0 (automatic) or 1 .. 4096");
    ctx->star_split = split;
    return MLENS_OK;
}

int mlens_star_split_for(const mlens_ctx *ctx, const mlens_grid *rays, int32_t *split_out)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    if (!split_out) return fail(MLENS_ERR_ARG, "split_out is NULL");
    int rc;
    if ((rc = check_rays(rays))) return rc;
    *split_out = effective_split(ctx, make_ray_grid(*rays));
    return MLENS_OK;
}

int mlens_shoot(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev, uint32_t flags,
                mlens_stats *stats_host, void *stream)
{
    return shoot_impl(ctx, rays, src, counts_dev, nullptr, flags, stats_host, stream);
}

int mlens_shoot_beta(mlens_ctx *ctx, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                     void *beta_dev, uint32_t flags, mlens_stats *stats_host, void *stream)
{
    if (!beta_dev) return fail(MLENS_ERR_ARG, "beta_dev is NULL");
    return shoot_impl(ctx, rays, src, counts_dev, beta_dev, flags, stats_host, stream);
}

int mlens_shoot_rows(mlens_ctx *ctx, const mlens_grid *rays, int32_t row_begin, int32_t row_end,
                     const mlens_grid *src, uint32_t *counts_dev, void *beta_dev, uint32_t flags,
                     mlens_stats *stats_host, void *stream)
{
    if (rays && row_begin == 0 && row_end == 0) row_end = rays->ny;
    return shoot_impl(ctx, rays, src, counts_dev, beta_dev, flags, stats_host, stream, row_begin, row_end);
}

int mlens_trace(mlens_ctx *ctx, const double *theta, int64_t k, double *beta, void *stream)
{
    if (!ctx) return fail(MLENS_ERR_ARG, "context is NULL");
    if (k < 0 || k >= (int64_t(1) << 36)) return fail(MLENS_ERR_ARG, "k must satisfy 0 <= k < 2^36");
    if (k == 0) return MLENS_OK;
    if (!theta || !beta) return fail(MLENS_ERR_ARG, "theta_host and beta_host must be non-NULL");
    int rc;
    if ((rc = check_current_device(ctx->device))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *d = nullptr;
    MLENS_CUDA(dmalloc(&d, (size_t)k * 2 * sizeof(double2)), "cudaMalloc(trace)");
    cudaError_t e = cudaMemcpyAsync(d, theta, (size_t)k * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_trace_fp64(ctx->d_stars, ctx->n_pad, ctx->lens, d, d + k, k, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(beta, d + k, (size_t)k * sizeof(double2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(d);
    if (e != cudaSuccess) return cuda_fail(e, "mlens_trace");
    return MLENS_OK;
}

int mlens_bin(const void *beta_dev, int64_t n, const mlens_grid *src, uint32_t *counts_dev, uint32_t flags,
              mlens_stats *stats_host, void *stream)
{
    if (n < 0 || n >= (int64_t(1) << 40)) return fail(MLENS_ERR_ARG, "n must satisfy 0 <= n < 2^40");
    return bin_impl(beta_dev, n, 0, 0, src, counts_dev, flags, stats_host, stream);
}

int mlens_bin_grid(const void *beta_dev, const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                   uint32_t flags, mlens_stats *stats_host, void *stream)
{
    int rc;
    if ((rc = check_rays(rays))) return rc;
    return bin_impl(beta_dev, (int64_t)rays->nx * rays->ny, rays->nx, rays->ny, src, counts_dev, flags, stats_host,
                    stream);
}

void mlens_destroy(mlens_ctx *ctx)
{
    if (!ctx) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (ctx->device >= 0 && prev != ctx->device) cudaSetDevice(ctx->device);
    if (ctx->d_stars || ctx->d_stats) cudaDeviceSynchronize();
    mlens_free_far_field(ctx);
    if (ctx->d_stars) dfree(ctx->d_stars);
    if (ctx->d_stats) dfree(ctx->d_stats);
    if (ctx->d_gpart) dfree(ctx->d_gpart);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    delete ctx;
}

}  // extern "C"
