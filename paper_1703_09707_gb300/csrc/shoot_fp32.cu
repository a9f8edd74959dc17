// shoot_fp32.cu -- the FP32 direct-sum ray-shooting kernels (Algorithm 1 with
// the deflection of Eq. 3 and the source position of Eq. 2), fused with the
// binning step, for one field (a grid of tiles) and for many fields (one
// persistent launch over a work queue of (field, tile) items).
//
// One CTA of 256 threads owns a 64 x (8*NP) tile of the ray grid; each thread
// owns 2*NP rays of one grid column, processed as NP packed pairs with the
// Blackwell f32x2 instructions (FADD2/FMUL2/FFMA2), so one instruction serves
// two rays.  Stars stream through shared memory in stages of SC; each stage is
// re-centred on the tile (star minus tile centre, once per star per CTA) and
// stored duplicated as (-dx,-dx,-dy,-dy),(m,m) so that a single broadcast
// LDS.128 + LDS.64 feeds every packed pair.  Per star and ray the work is
// FADD, FFMA (r^2), MUFU.RCP, FMUL (m/r^2), 2 FFMA (accumulate): the MUFU
// reciprocal (16 per SM per clock) is the only unit near saturation.
//
// Precision (MLENS_PREC_FP32): rays and stars are relative to an FP32 tile
// centre c, so differences of nearby positions carry no absolute-coordinate
// rounding.  Terms are accumulated in plain FP32 over 32 stars and each 32-star
// partial is added to the running sum with Kahan compensation.  The
// smooth+shear part A c of the tile centre is formed in FP64 once per tile, and
// beta = A c + A delta - S is assembled as a float pair, so the only rounding
// left at the full coordinate scale is the exact binning rule's.  The stage
// size SC does not change the arithmetic (the 32-star chunks are the same), the
// tile shape NP does (it moves the tile centres).
// MLENS_PREC_FP32_NAIVE keeps absolute coordinates and one running FP32 sum
// (Algorithm 1 written in single precision).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "tile.cuh"

namespace mlens {

template <int NP, int SC, bool NAIVE, int NRP>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_fp32(ShootArgs a, int by0)
{
    __shared__ __align__(16) ShootSmem<SC> sm;
    __shared__ TileShared ts;
    shoot_tile<NP, SC, NAIVE, NRP>(a, blockIdx.x, by0 + (int)blockIdx.y, sm, ts);
}

// Split star sum: clusters of SPLIT CTAs along x share one tile (tile column
// blockIdx.x / SPLIT); partials are reduced through distributed shared memory.
template <int NP, int SPLIT>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_split(ShootArgs a, int by0)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    extern __shared__ float4 part[];  // 2 NP float4 per thread
    shoot_tile<NP, kSplitStage, false, 0, SPLIT>(a, (int)(blockIdx.x / SPLIT), by0 + (int)blockIdx.y, sm, ts, part);
}

// Split star sum through global memory: CTA (tile column blockIdx.x / R, slice
// blockIdx.x % R) sums one slice of the stars and stores its partials; tile rows
// from `ty_base` on are numbered from 0 in the partials.
template <int NP>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_slices(ShootArgs a, int by0, int ty_base)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    const int R = a.gslices, tiles_x = (a.rays.nx + kTileX - 1) / kTileX;
    const int bx = (int)(blockIdx.x / R), r = (int)(blockIdx.x % R), by = by0 + (int)blockIdx.y;
    shoot_tile<NP, kSplitStage, false, 0, 1, 0, 1>(a, bx, by, sm, ts, nullptr, (int64_t)(by - ty_base) * tiles_x + bx,
                                                    r);
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

// Persistent kernel over many fields: CTAs pull (field, tile) items from one
// atomic counter until the queue is empty.  Items are numbered field by field in
// the order `order` (heaviest field first, so the tail is made of light items);
// begin[k] is the first item of the k-th field in that order (begin[nf] = total).
template <int NP, int SC, int NRP>
__global__ void __launch_bounds__(kThreads, 2)
    k_shoot_batch(const ShootArgs *fields, const int *order, const int64_t *begin, int nf, int64_t total,
                  unsigned long long *counter)
{
    __shared__ __align__(16) ShootSmem<SC> sm;
    __shared__ TileShared ts;
    __shared__ long long s_item;
    for (;;) {
        __syncthreads();  // everyone has finished with the previous item number
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (begin[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const ShootArgs &A = fields[order[lo]];
        const int64_t t = item - begin[lo];
        const int tiles_x = (A.rays.nx + kTileX - 1) / kTileX;
        shoot_tile<NP, SC, false, NRP>(A, (int)(t % tiles_x), (int)(t / tiles_x), sm, ts);
    }
}

// Tile rows [ty0, ty1) of the grid; ty1 < 0 means through the last tile row.
static inline int tile_row_end(const ShootArgs &a, int np, int ty1)
{
    const int ty = (a.rays.ny + tile_rows(np) - 1) / tile_rows(np);
    return ty1 < 0 || ty1 > ty ? ty : ty1;
}

template <int NP, int SC, bool NAIVE, int NRP>
static cudaError_t launch_t(const ShootArgs &a, cudaStream_t s, int ty0, int ty1)
{
    // tile rows in launches of at most 65535 (the grid's y limit)
    const int tx = (a.rays.nx + kTileX - 1) / kTileX, ty = tile_row_end(a, NP, ty1);
    for (int by0 = ty0; by0 < ty; by0 += 65535) {
        const dim3 grid((unsigned)tx, (unsigned)min(65535, ty - by0));
        k_shoot_fp32<NP, SC, NAIVE, NRP><<<grid, kThreads, 0, s>>>(a, by0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool NAIVE, int NRP>
static cudaError_t launch_sel(const ShootArgs &a, int np, int sc, cudaStream_t s, int ty0, int ty1)
{
    if (np == 2) {
        if (sc == 128) return launch_t<2, 128, NAIVE, NRP>(a, s, ty0, ty1);
        if (sc == 512) return launch_t<2, 512, NAIVE, NRP>(a, s, ty0, ty1);
        return launch_t<2, 256, NAIVE, NRP>(a, s, ty0, ty1);
    }
    if (sc == 128) return launch_t<4, 128, NAIVE, NRP>(a, s, ty0, ty1);
    if (sc == 512) return launch_t<4, 512, NAIVE, NRP>(a, s, ty0, ty1);
    return launch_t<4, 256, NAIVE, NRP>(a, s, ty0, ty1);
}

cudaError_t launch_shoot_fp32(const ShootArgs &a, int pairs_per_thread, bool naive, cudaStream_t s, int stage,
                              int fma_pairs, int ty0, int ty1)
{
    if (naive) return launch_sel<true, 0>(a, pairs_per_thread, stage, s, ty0, ty1);
    return fma_pairs ? launch_sel<false, 1>(a, pairs_per_thread, stage, s, ty0, ty1)
                     : launch_sel<false, 0>(a, pairs_per_thread, stage, s, ty0, ty1);
}

template <int NP, int SPLIT>
static cudaError_t launch_split_t(const ShootArgs &a, cudaStream_t s, int ty0, int ty1)
{
    const int tx = (a.rays.nx + kTileX - 1) / kTileX, ty = tile_row_end(a, NP, ty1);
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
    cudaError_t e0 = cudaFuncSetAttribute(k_shoot_split<NP, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)cfg.dynamicSmemBytes);
    // two CTAs of ~49 KB per SM: ask for the largest shared-memory carveout
    if (e0 == cudaSuccess)
        e0 = cudaFuncSetAttribute(k_shoot_split<NP, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared);
    if (e0 != cudaSuccess) return e0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int by0 = ty0; by0 < ty; by0 += 65535) {
        cfg.gridDim = dim3((unsigned)(tx * SPLIT), (unsigned)min(65535, ty - by0));
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_shoot_split<NP, SPLIT>, a, by0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The split star sum over a list of tiles (tile = by * tiles_x + bx), one
// cluster per listed tile: the learned far field's fallback tiles.
template <int SPLIT>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_split_list(ShootArgs a, const int *tiles)
{
    __shared__ __align__(16) ShootSmem<kSplitStage> sm;
    __shared__ TileShared ts;
    extern __shared__ float4 part[];  // 2 NP float4 per thread
    const int ntx = (a.rays.nx + kTileX - 1) / kTileX;
    const int t = tiles[blockIdx.x / SPLIT];
    shoot_tile<4, kSplitStage, false, 0, SPLIT>(a, t % ntx, t / ntx, sm, ts, part);
}

template <int SPLIT>
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
    cudaError_t e = cudaFuncSetAttribute(k_shoot_split_list<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.dynamicSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_shoot_split_list<SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3((unsigned)(ntiles * SPLIT));
    return cudaLaunchKernelEx(&cfg, k_shoot_split_list<SPLIT>, a, tiles);
}

cudaError_t launch_shoot_split_list(const ShootArgs &a, const int *tiles, int64_t ntiles, int split, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles * split > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (split == 2) return launch_split_list_t<2>(a, tiles, ntiles, s);
    if (split == 4) return launch_split_list_t<4>(a, tiles, ntiles, s);
    if (split == 8) return launch_split_list_t<8>(a, tiles, ntiles, s);
    return cudaErrorInvalidValue;
}

int fallback_star_split(int64_t nstars)
{
    for (int R = 8; R >= 2; R /= 2)
        if (nstars / R >= kMinSplitStars) return R;
    return 1;
}

template <int NP>
static cudaError_t launch_split_np(const ShootArgs &a, int split, cudaStream_t s, int ty0, int ty1)
{
    switch (split) {
    case 2: return launch_split_t<NP, 2>(a, s, ty0, ty1);
    case 3: return launch_split_t<NP, 3>(a, s, ty0, ty1);
    case 4: return launch_split_t<NP, 4>(a, s, ty0, ty1);
    case 5: return launch_split_t<NP, 5>(a, s, ty0, ty1);
    case 6: return launch_split_t<NP, 6>(a, s, ty0, ty1);
    case 7: return launch_split_t<NP, 7>(a, s, ty0, ty1);
    case 8: return launch_split_t<NP, 8>(a, s, ty0, ty1);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_shoot_split(const ShootArgs &a, int pairs_per_thread, int split, cudaStream_t s, int ty0, int ty1)
{
    return pairs_per_thread == 2 ? launch_split_np<2>(a, split, s, ty0, ty1) : launch_split_np<4>(a, split, s, ty0, ty1);
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

template <int NP>
static cudaError_t launch_gsplit_t(const ShootArgs &a0, int split, float4 *part, int rows_per_pass, cudaStream_t s,
                                   int ty0, int ty1)
{
    ShootArgs a = a0;
    a.gpart = part;
    a.gslices = split;
    const int tx = (a.rays.nx + kTileX - 1) / kTileX, ty = tile_row_end(a, NP, ty1);
    // static shared memory only (two CTAs of ~17 KB per SM): the largest carveout
    cudaError_t e = cudaFuncSetAttribute(k_shoot_slices<NP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if ((int64_t)tx * split > 0x7fffffff) return cudaErrorInvalidConfiguration;
    // one pass per rows_per_pass tile rows: the slices, then their fold (same stream,
    // so the next pass's slices overwrite partials the fold has read)
    for (int by0 = ty0; by0 < ty; by0 += rows_per_pass) {
        const int rows = std::min(rows_per_pass, ty - by0);
        k_shoot_slices<NP><<<dim3((unsigned)(tx * split), (unsigned)rows), kThreads, 0, s>>>(a, by0, by0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_fold_slices<NP><<<dim3((unsigned)tx, (unsigned)rows), kThreads, 0, s>>>(a, by0, by0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_shoot_gsplit(const ShootArgs &a, int pairs_per_thread, int split, float4 *part, int rows_per_pass,
                                cudaStream_t s, int ty0, int ty1)
{
    if (split < 2 || split > kMaxSplit || !part || rows_per_pass < 1 || rows_per_pass > 65535)
        return cudaErrorInvalidValue;
    return pairs_per_thread == 2 ? launch_gsplit_t<2>(a, split, part, rows_per_pass, s, ty0, ty1)
                                 : launch_gsplit_t<4>(a, split, part, rows_per_pass, s, ty0, ty1);
}

int64_t tiles_of(const RayGrid &r, int pairs_per_thread)
{
    const int ty = tile_rows(pairs_per_thread);
    return (int64_t)((r.nx + kTileX - 1) / kTileX) * (int64_t)((r.ny + ty - 1) / ty);
}

template <int NP, int SC, int NRP>
static cudaError_t grid_b(int *grid)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shoot_batch<NP, SC, NRP>, kThreads, 0);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *grid = nsm * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

template <int NRP>
static cudaError_t grid_sel(int np, int sc, int *grid)
{
    if (np == 2) {
        if (sc == 128) return grid_b<2, 128, NRP>(grid);
        if (sc == 512) return grid_b<2, 512, NRP>(grid);
        return grid_b<2, 256, NRP>(grid);
    }
    if (sc == 128) return grid_b<4, 128, NRP>(grid);
    if (sc == 512) return grid_b<4, 512, NRP>(grid);
    return grid_b<4, 256, NRP>(grid);
}

cudaError_t batch_grid_size(int pairs_per_thread, int stage, int *grid, int fma_pairs)
{
    return fma_pairs ? grid_sel<1>(pairs_per_thread, stage, grid) : grid_sel<0>(pairs_per_thread, stage, grid);
}

template <int NP, int SC, int NRP>
static cudaError_t launch_b(const BatchLaunch &b, cudaStream_t s)
{
    const int64_t want = b.grid > 0 ? b.grid : 1;
    const unsigned grid = (unsigned)(b.total < want ? (b.total > 0 ? b.total : 1) : want);
    k_shoot_batch<NP, SC, NRP><<<grid, kThreads, 0, s>>>(b.fields, b.order, b.begin, b.nfields, b.total, b.counter);
    return cudaGetLastError();
}

template <int NRP>
static cudaError_t launch_bsel(const BatchLaunch &b, int np, int sc, cudaStream_t s)
{
    if (np == 2) {
        if (sc == 128) return launch_b<2, 128, NRP>(b, s);
        if (sc == 512) return launch_b<2, 512, NRP>(b, s);
        return launch_b<2, 256, NRP>(b, s);
    }
    if (sc == 128) return launch_b<4, 128, NRP>(b, s);
    if (sc == 512) return launch_b<4, 512, NRP>(b, s);
    return launch_b<4, 256, NRP>(b, s);
}

cudaError_t launch_shoot_batch(const BatchLaunch &b, int pairs_per_thread, int stage, cudaStream_t s, int fma_pairs)
{
    return fma_pairs ? launch_bsel<1>(b, pairs_per_thread, stage, s) : launch_bsel<0>(b, pairs_per_thread, stage, s);
}

}  // namespace mlens
