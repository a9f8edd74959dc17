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
