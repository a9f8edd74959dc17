// noalloc.cu -- mlens_shoot_noalloc: the FP32 shooting kernel for callers that
// cannot allocate device memory (host applications that own all device
// allocations, real-time loops that must stay out of the allocator).  Its working
// memory is one file-scope device array: a padded copy of the caller's stars and
// the ray counters.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>

#include "mlens_internal.h"

namespace mlens {
namespace {

constexpr int64_t kNoAllocStars = MLENS_NOALLOC_MAX_STARS;
constexpr int64_t kNoAllocCap = kNoAllocStars + kStarPad;

struct NoAllocScratch {
    float4 stars[kNoAllocCap];        // caller's stars, padded to a multiple of kStarPad
    unsigned long long stats[4];      // [binned, out, nan, unused]
};

// The working memory.  Host code must not use this name as a pointer: on the host it
// is only a stand-in, and the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
// device address per device ordinal, set on the first call on that device and
// kept for the life of the process (a device reset is not followed)
NoAllocScratch *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

__global__ void k_noalloc_stage(const float4 *in, int64_t n, int64_t npad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += stride)
        g_noalloc_scratch.stars[i] = i < n ? in[i] : make_float4(kPadCoord, kPadCoord, 0.0f, 0.0f);
    if (blockIdx.x == 0 && threadIdx.x < 4) g_noalloc_scratch.stats[threadIdx.x] = 0ull;
}

int arg_error(const char *msg)
{
    set_last_error(msg);
    return MLENS_ERR_ARG;
}

int cuda_error(cudaError_t e, const char *what)
{
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    clear_pending_error();
    return MLENS_ERR_CUDA;
}

bool box_ok(const mlens_grid *g)
{
    return g && std::isfinite(g->x0) && std::isfinite(g->x1) && std::isfinite(g->y0) && std::isfinite(g->y1) &&
           g->x1 > g->x0 && g->y1 > g->y0 && g->nx >= 1 && g->ny >= 1;
}

// Device address of the working memory on the current device (looked up once per device).
int scratch_address(NoAllocScratch **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return arg_error("device ordinal beyond the no-alloc table");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc working memory)");
        g_scratch_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    return MLENS_OK;
}

}  // namespace
}  // namespace mlens

using namespace mlens;

extern "C" int mlens_shoot_noalloc(const void *stars_dev, int64_t n, double kappa_c, double gamma1, double gamma2,
                                   const mlens_grid *rays, const mlens_grid *src, uint32_t *counts_dev,
                                   uint32_t flags, mlens_stats *stats_host, void *stream)
{
    if (n < 0 || n > kNoAllocStars)
        return arg_error("mlens_shoot_noalloc: n must satisfy 0 <= n <= MLENS_NOALLOC_MAX_STARS (65536)");
    if (n > 0 && !stars_dev) return arg_error("mlens_shoot_noalloc: stars_dev is NULL");
    if (((uintptr_t)stars_dev & 15u) != 0) return arg_error("mlens_shoot_noalloc: stars_dev must be 16-byte aligned");
    if (!std::isfinite(kappa_c) || !std::isfinite(gamma1) || !std::isfinite(gamma2))
        return arg_error("mlens_shoot_noalloc: kappa_c and gamma must be finite");
    if (!box_ok(rays) || rays->nx > (1 << 20) || rays->ny > (1 << 20))
        return arg_error("mlens_shoot_noalloc: bad rays grid (finite box, 1 <= nx, ny <= 2^20)");
    if (!box_ok(src) || (int64_t)src->nx * src->ny > (int64_t(1) << 30))
        return arg_error("mlens_shoot_noalloc: bad source grid (finite box, nx*ny <= 2^30)");
    if (!counts_dev || ((uintptr_t)counts_dev & 3u) != 0)
        return arg_error("mlens_shoot_noalloc: counts_dev must be non-NULL and 4-byte aligned");
    if (flags & ~MLENS_ACCUMULATE) return arg_error("mlens_shoot_noalloc: unknown flag bits");

    NoAllocScratch *sc = nullptr;
    int rc = scratch_address(&sc);
    if (rc != MLENS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npad = (n + kStarPad - 1) / kStarPad * kStarPad;
    cudaError_t e;
    if (!(flags & MLENS_ACCUMULATE)) {
        e = cudaMemsetAsync(counts_dev, 0, (size_t)src->nx * (size_t)src->ny * sizeof(uint32_t), s);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(counts)");
    }
    const int64_t blocks = npad > 0 ? (npad + 255) / 256 : 1;
    k_noalloc_stage<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float4 *>(stars_dev), n, npad);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "no-alloc staging kernel launch");

    ShootArgs a{};
    a.stars = sc->stars;
    a.nstars = npad;
    a.rays = make_ray_grid(*rays);
    a.bin = make_bin_grid(*src);
    a.lens = make_lens_terms(kappa_c, gamma1, gamma2);
    a.counts = counts_dev;
    a.stats = sc->stats;
    a.beta_out = nullptr;
    if ((e = launch_shoot_fp32(a, 4, false, s, 256, kDefaultFmaPairs)) != cudaSuccess)
        return cuda_error(e, "no-alloc shoot kernel launch");
    if (stats_host) {
        unsigned long long h[3];
        if ((e = cudaMemcpyAsync(h, sc->stats, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync(no-alloc counters)");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
        stats_host->rays_total = (uint64_t)rays->nx * (uint64_t)rays->ny;
        stats_host->rays_binned = h[0];
        stats_host->rays_out = h[1];
        stats_host->rays_nan = h[2];
    }
    return MLENS_OK;
}
