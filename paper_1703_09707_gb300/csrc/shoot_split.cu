// shoot_split.cu -- the split star sum (the closing discussion of very large star
// fields: one image position's bending-angle sum shared by several threads).  The
// stars are cut into consecutive 32-aligned slices, one CTA per slice of a ray
// tile, and the slices' compensated partial sums are folded in slice order before
// beta and binning: through distributed shared memory within a thread-block
// cluster (2 .. 8 CTAs), or through global memory and a second kernel (9 .. 4096
// CTAs).  Also the automatic choice of the split, and the learned far field's
// fallback tiles (a list of tiles, one cluster each).  NRP: the reciprocal split
// of tile.cuh (0: MUFU alone; 1: a share on the FMA pipe).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "tile.cuh"

namespace mlens {

// Tile rows [ty0, ty1) of the grid; ty1 < 0 means through the last tile row.
static inline int tile_row_end_s(const ShootArgs &a, int np, int ty1)
{
    const int ty = (a.rays.ny + tile_rows(np) - 1) / tile_rows(np);
    return ty1 < 0 || ty1 > ty ? ty : ty1;
}

// Split star sum: clusters of SPLIT CTAs along x share one tile (tile column
// blockIdx.x / SPLIT); partials are reduced through distributed shared memory.
template <int NP, int SPLIT, int NRP>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_split(ShootArgs a, int by0)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    extern __shared__ float4 part[];  // 2 NP float4 per thread
    shoot_tile<NP, kSplitStage, false, NRP, SPLIT>(a, (int)(blockIdx.x / SPLIT), by0 + (int)blockIdx.y, sm, ts, part);
}

// Split star sum through global memory: CTA (tile column blockIdx.x / R, slice
// blockIdx.x % R) sums one slice of the stars and stores its partials; tile rows
// from `ty_base` on are numbered from 0 in the partials.
template <int NP, int NRP>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_slices(ShootArgs a, int by0, int ty_base)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    const int R = a.gslices, tiles_x = (a.rays.nx + kTileX - 1) / kTileX;
    const int bx = (int)(blockIdx.x / R), r = (int)(blockIdx.x % R), by = by0 + (int)blockIdx.y;
    shoot_tile<NP, kSplitStage, false, NRP, 1, 0, 1>(a, bx, by, sm, ts, nullptr,
                                                      (int64_t)(by - ty_base) * tiles_x + bx, r);
}

// ... and the tile's partials folded in slice order, then beta and binning.
template <int NP>
__global__ void __launch_bounds__(kThreads, 2) k_fold_slices(ShootArgs a, int by0, int ty_base)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    const int tiles_x = (a.rays.nx + kTileX - 1) / kTileX;
    const int bx = (int)blockIdx.x, by = by0 + (int)blockIdx.y;
    shoot_tile<NP, kSplitStage, false, 0, 1, 0, 2>(a, bx, by, sm, ts, nullptr, (int64_t)(by - ty_base) * tiles_x + bx);
}

template <int NP, int SPLIT, int NRP>
static cudaError_t launch_split_t(const ShootArgs &a, cudaStream_t s, int ty0, int ty1)
{
    const int tx = (a.rays.nx + kTileX - 1) / kTileX, ty = tile_row_end_s(a, NP, ty1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SPLIT;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 2 * NP * kThreads * sizeof(float4);
    // static (the stage/window union) + dynamic (partials) exceeds the 48 KB a
    // launch gets without opting in for NP = 4
    cudaError_t e0 = cudaFuncSetAttribute(k_shoot_split<NP, SPLIT, NRP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)cfg.dynamicSmemBytes);
    // two CTAs of ~49 KB per SM: ask for the largest shared-memory carveout
    if (e0 == cudaSuccess)
        e0 = cudaFuncSetAttribute(k_shoot_split<NP, SPLIT, NRP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared);
    if (e0 != cudaSuccess) return e0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int by0 = ty0; by0 < ty; by0 += 65535) {
        cfg.gridDim = dim3((unsigned)(tx * SPLIT), (unsigned)min(65535, ty - by0));
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_shoot_split<NP, SPLIT, NRP>, a, by0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The split star sum over a list of tiles (tile = by * tiles_x + bx), one
// cluster per listed tile: the learned far field's fallback tiles.
template <int SPLIT, int NRP>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_split_list(ShootArgs a, const int *tiles)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    extern __shared__ float4 part[];  // 2 NP float4 per thread
    const int ntx = (a.rays.nx + kTileX - 1) / kTileX;
    const int t = tiles[blockIdx.x / SPLIT];
    shoot_tile<4, kSplitStage, false, NRP, SPLIT>(a, t % ntx, t / ntx, sm, ts, part);
}

template <int SPLIT, int NRP>
static cudaError_t launch_split_list_t(const ShootArgs &a, const int *tiles, int64_t ntiles, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = SPLIT;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 2 * 4 * kThreads * sizeof(float4);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaFuncSetAttribute(k_shoot_split_list<SPLIT, NRP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.dynamicSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_shoot_split_list<SPLIT, NRP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3((unsigned)(ntiles * SPLIT));
    return cudaLaunchKernelEx(&cfg, k_shoot_split_list<SPLIT, NRP>, a, tiles);
}

template <int NRP>
static cudaError_t launch_split_list_r(const ShootArgs &a, const int *tiles, int64_t ntiles, int split, cudaStream_t s)
{
    if (split == 2) return launch_split_list_t<2, NRP>(a, tiles, ntiles, s);
    if (split == 4) return launch_split_list_t<4, NRP>(a, tiles, ntiles, s);
    if (split == 8) return launch_split_list_t<8, NRP>(a, tiles, ntiles, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_shoot_split_list(const ShootArgs &a, const int *tiles, int64_t ntiles, int split, cudaStream_t s,
                                    int fma_pairs)
{
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles * split > 0x7fffffff) return cudaErrorInvalidConfiguration;
    return fma_pairs ? launch_split_list_r<1>(a, tiles, ntiles, split, s)
                     : launch_split_list_r<0>(a, tiles, ntiles, split, s);
}

int fallback_star_split(int64_t nstars)
{
    for (int R = 8; R >= 2; R /= 2)
        if (nstars / R >= kMinSplitStars) return R;
    return 1;
}

template <int NP, int NRP>
static cudaError_t launch_split_np(const ShootArgs &a, int split, cudaStream_t s, int ty0, int ty1)
{
    switch (split) {
    case 2: return launch_split_t<NP, 2, NRP>(a, s, ty0, ty1);
    case 3: return launch_split_t<NP, 3, NRP>(a, s, ty0, ty1);
    case 4: return launch_split_t<NP, 4, NRP>(a, s, ty0, ty1);
    case 5: return launch_split_t<NP, 5, NRP>(a, s, ty0, ty1);
    case 6: return launch_split_t<NP, 6, NRP>(a, s, ty0, ty1);
    case 7: return launch_split_t<NP, 7, NRP>(a, s, ty0, ty1);
    case 8: return launch_split_t<NP, 8, NRP>(a, s, ty0, ty1);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_shoot_split(const ShootArgs &a, int pairs_per_thread, int split, cudaStream_t s, int ty0, int ty1,
                               int fma_pairs)
{
    if (pairs_per_thread == 2)
        return fma_pairs ? launch_split_np<2, 1>(a, split, s, ty0, ty1) : launch_split_np<2, 0>(a, split, s, ty0, ty1);
    return fma_pairs ? launch_split_np<4, 1>(a, split, s, ty0, ty1) : launch_split_np<4, 0>(a, split, s, ty0, ty1);
}

int auto_star_split(const RayGrid &r, int pairs_per_thread, int64_t nstars, int nsm)
{
    // One CTA per SM already keeps the SM's reciprocal unit near its peak, and
    // a second resident CTA (the kernels are launch-bounded to two per SM)
    // shares it.  For C = tiles * R equal CTAs of work T / R the map therefore
    // takes T / R when C <= nsm (one CTA per SM) and about
    // ceil(C / (2 nsm)) * 2 T / R otherwise (rounds of two CTAs at half speed).
    // The split through global memory takes R = the smallest number above
    // kMaxClusterSplit giving at least 16 CTAs per SM, so the last round is
    // nearly full; it is taken if it gains 5 % and leaves every slice
    // kMinSplitStars stars.  (Cluster splits are not chosen automatically: a
    // cluster needs all its CTAs free at once within one GPC, and on few-tile
    // grids that fragmentation cost as much as the split gained.)  With too few
    // stars for that many slices, the clusters of 2, 4 or 8 CTAs are weighed the
    // same way.
    const double tiles = (double)tiles_of(r, pairs_per_thread);
    const double sms = (double)(nsm > 0 ? nsm : 1);
    auto cost = [&](int64_t R) {
        const double c = tiles * (double)R;
        return c <= sms ? 1.0 / (double)R : std::ceil(c / (2.0 * sms)) * 2.0 / (double)R;
    };
    const double c1 = cost(1);
    int64_t rg = (int64_t)std::ceil(16.0 * sms / tiles);
    if (rg <= kMaxClusterSplit) rg = kMaxClusterSplit + 1;
    if (rg <= kMaxSplit && nstars / rg >= kMinSplitStars) return cost(rg) < c1 / 1.05 ? (int)rg : 1;
    int best = 1;
    double bc = c1;
    for (int R = 2; R <= kMaxClusterSplit; R *= 2) {
        if (nstars / R < kMinSplitStars) break;
        const double c = cost(R);
        if (c < bc / 1.05) {
            best = R;
            bc = c;
        }
    }
    return best;
}

// Partials of one pass: rows_per_pass tile rows x tiles_x tiles x split slices x
// 2 NP float4 per thread.
size_t gsplit_part_bytes(const RayGrid &r, int pairs_per_thread, int split, int tile_rows_per_pass)
{
    const size_t tiles_x = (size_t)((r.nx + kTileX - 1) / kTileX);
    return (size_t)tile_rows_per_pass * tiles_x * (size_t)split * (size_t)(2 * pairs_per_thread * kThreads) *
           sizeof(float4);
}

int gsplit_rows_per_pass(const RayGrid &r, int pairs_per_thread, int split, size_t bytes)
{
    const size_t one = gsplit_part_bytes(r, pairs_per_thread, split, 1);
    const int ty = (int)((r.ny + tile_rows(pairs_per_thread) - 1) / tile_rows(pairs_per_thread));
    const size_t k = bytes / one;
    return (int)std::max<size_t>(1, std::min<size_t>(k, (size_t)std::min(ty, 65535)));
}

template <int NP, int NRP>
static cudaError_t launch_gsplit_t(const ShootArgs &a0, int split, float4 *part, int rows_per_pass, cudaStream_t s,
                                   int ty0, int ty1)
{
    ShootArgs a = a0;
    a.gpart = part;
    a.gslices = split;
    const int tx = (a.rays.nx + kTileX - 1) / kTileX, ty = tile_row_end_s(a, NP, ty1);
    // static shared memory only (two CTAs of ~17 KB per SM): the largest carveout
    cudaError_t e = cudaFuncSetAttribute(k_shoot_slices<NP, NRP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if ((int64_t)tx * split > 0x7fffffff) return cudaErrorInvalidConfiguration;
    // one pass per rows_per_pass tile rows: the slices, then their fold (same stream,
    // so the next pass's slices overwrite partials the fold has read)
    for (int by0 = ty0; by0 < ty; by0 += rows_per_pass) {
        const int rows = std::min(rows_per_pass, ty - by0);
        k_shoot_slices<NP, NRP><<<dim3((unsigned)(tx * split), (unsigned)rows), kThreads, 0, s>>>(a, by0, by0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_fold_slices<NP><<<dim3((unsigned)tx, (unsigned)rows), kThreads, 0, s>>>(a, by0, by0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_shoot_gsplit(const ShootArgs &a, int pairs_per_thread, int split, float4 *part, int rows_per_pass,
                                cudaStream_t s, int ty0, int ty1, int fma_pairs)
{
    if (split < 2 || split > kMaxSplit || !part || rows_per_pass < 1 || rows_per_pass > 65535)
        return cudaErrorInvalidValue;
    if (pairs_per_thread == 2)
        return fma_pairs ? launch_gsplit_t<2, 1>(a, split, part, rows_per_pass, s, ty0, ty1)
                         : launch_gsplit_t<2, 0>(a, split, part, rows_per_pass, s, ty0, ty1);
    return fma_pairs ? launch_gsplit_t<4, 1>(a, split, part, rows_per_pass, s, ty0, ty1)
                     : launch_gsplit_t<4, 0>(a, split, part, rows_per_pass, s, ty0, ty1);
}

}  // namespace mlens
