// mlens_internal.h -- host-side structures shared by the translation units of
// libmlens (not part of the public ABI; see include/mlens.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mlens.h"

namespace mlens {

// Stars are padded on the device to a multiple of this many records (one
// compensated-summation chunk) with massless stars far away; they add exactly
// zero to every sum.
constexpr int kStarPad = 32;
constexpr float kPadCoord = 1.0e15f;

// Float-pair constants of one source-map axis: x0 = x0h + x0l and
// s = n / (x1 - x0) = sh + sl, each split from its double value.
struct AxisPair {
    float x0h, x0l, sh, sl;
    float sh2;  // 2 |sh|
    float tq;   // 2 |x0l| |sh| + 2^-100, rounded up: the constant part of the quick test's bound
    int n;
};

struct BinGrid {
    AxisPair ax, ay;
    double x0, x1, y0, y1;  // the double box, for the FP64 rule
    int nx, ny;
};

// Ray grid with its spacing split into float pairs.
struct RayGrid {
    double x0, x1, y0, y1;
    int nx, ny;
    double dx, dy;          // (x1-x0)/nx, (y1-y0)/ny
    float dxh, dxl, dyh, dyl;
    double qx, qy, qxinv, qyinv;  // largest powers of two <= dx, dy (tile-centre quantum) and inverses
    int lo;                 // 1: ray offsets from the tile centres need a low part (see make_ray_grid)
};

// Smooth + shear part of Eq. (1): beta = A theta - star sum, A = I - M,
// M = [[kc+g1, g2], [g2, kc-g1]].
struct LensTerms {
    double kc, g1, g2;
    double a11, a12, a22;   // A in double
    float fa11, fa12, fa22; // A rounded to float
    float fm11, fm12, fm22; // M rounded to float (naive variant)
};

struct ShootArgs {
    const float4 *stars;    // (x, y, m, 0), padded
    int64_t nstars;         // padded count, multiple of kStarPad
    RayGrid rays;
    BinGrid bin;
    LensTerms lens;
    uint32_t *counts;
    unsigned long long *stats;  // [binned, out, nan]
    void *beta_out;         // nullable: float4 pairs or double2 (FP64)
    float4 *gpart;          // global split: 2 NP float4 per thread per (tile, slice) (launch_shoot_gsplit)
    int gslices;            // global split: slices per tile
};

struct BinArgs {
    const float4 *beta;
    int64_t n;
    int rnx, rny;  // records form a row-major rnx x rny ray grid (0 = flat order)
    BinGrid bin;
    uint32_t *counts;
    unsigned long long *stats;
};

// Persistent multi-field launch: device tables built by the batch API.
struct BatchLaunch {
    int grid;                     // persistent CTAs (SMs x resident CTAs per SM)
    const ShootArgs *fields;      // nfields descriptors (device)
    const int *order;             // field processing order, heaviest first (device)
    const int64_t *begin;         // nfields+1 item offsets in that order (device)
    int nfields;
    int64_t total;                // total (field, tile) items
    unsigned long long *counter;  // work-queue counter, zero before each launch (device)
};

// launchers (defined in the .cu files)
// pairs_per_thread in {2, 4} (4 or 8 rays per thread); stage in {128, 256, 512} stars
// fma_pairs in {0, 1}: 1 takes a share of the reciprocals (pair 0 on every third
// star, 7.8 %) from the FMA pipe, 0 every reciprocal from the MUFU unit
// [ty0, ty1): the tile rows to shoot (tile_rows(pairs_per_thread) ray rows each;
// ty1 < 0 = through the last)
cudaError_t launch_shoot_fp32(const ShootArgs &a, int pairs_per_thread, bool naive, cudaStream_t s,
                              int stage = 256, int fma_pairs = 0, int ty0 = 0, int ty1 = -1);
cudaError_t launch_shoot_batch(const BatchLaunch &b, int pairs_per_thread, int stage, cudaStream_t s,
                               int fma_pairs = 0);
cudaError_t batch_grid_size(int pairs_per_thread, int stage, int *grid, int fma_pairs = 0);
int64_t tiles_of(const RayGrid &r, int pairs_per_thread);
// ray rows [row0, row1) (row0 a multiple of 4; row1 < 0 = through the last)
cudaError_t launch_shoot_fp64(const ShootArgs &a, cudaStream_t s, int row0 = 0, int row1 = -1);
cudaError_t launch_trace_fp64(const float4 *stars, int64_t nstars, const LensTerms &lens, const double2 *theta,
                              double2 *beta, int64_t k, cudaStream_t s);
// Split star sum (shoot_split.cu; re-centred FP32, 256-star stages, either
// reciprocal split): clusters of `split` in 2 .. 8 CTAs per tile.  auto_star_split
// picks the split for a grid (1 = none) from the wave efficiency on `nsm` SMs.
constexpr int kSplitStage = 256;
constexpr int64_t kMinSplitStars = 2048;
cudaError_t launch_shoot_split(const ShootArgs &a, int pairs_per_thread, int split, cudaStream_t s, int ty0, int ty1,
                               int fma_pairs);
int auto_star_split(const RayGrid &r, int pairs_per_thread, int64_t nstars, int nsm);
// The split star sum through global memory (splits above kMaxClusterSplit): each of
// `split` CTAs per tile sums one slice of the stars and stores its partials in
// `part` (a workspace of gsplit_part_bytes); a second kernel folds them in slice
// order and bins.  Tile rows go in passes of rows_per_pass (gsplit_rows_per_pass for
// a workspace of `bytes`).
constexpr int kMaxClusterSplit = 8;
constexpr int kDefaultFmaPairs = 1;  // the reciprocal split a context and the no-allocation entry start with
constexpr int kMaxSplit = 4096;
size_t gsplit_part_bytes(const RayGrid &r, int pairs_per_thread, int split, int tile_rows_per_pass);
int gsplit_rows_per_pass(const RayGrid &r, int pairs_per_thread, int split, size_t bytes);
cudaError_t launch_shoot_gsplit(const ShootArgs &a, int pairs_per_thread, int split, float4 *part, int rows_per_pass,
                                cudaStream_t s, int ty0, int ty1, int fma_pairs);
// Tiles of a list (tile = by * tiles_x + bx; 8 rays per thread), one cluster of
// `split` CTAs per tile; fallback_star_split is the split used for the learned
// far field's fallback tiles: the largest of 8, 4, 2 leaving kMinSplitStars
// stars per slice, else 1 (no split).
cudaError_t launch_shoot_split_list(const ShootArgs &a, const int *tiles, int64_t ntiles, int split, cudaStream_t s,
                                    int fma_pairs);
int fallback_star_split(int64_t nstars);
cudaError_t launch_bin(const BinArgs &a, cudaStream_t s);

// helpers (api.cu)
void set_last_error(const std::string &msg);
// A failed launch (a bad configuration, an exhausted resource) leaves its error
// pending in the runtime; the next launch's cudaGetLastError would report it
// again.  Every error path clears it after recording the message (errors that
// corrupt the context stay sticky regardless).
inline void clear_pending_error() { (void)cudaGetLastError(); }
// Every device allocation of the library goes through these: they keep count of
// the bytes in use and refuse (cudaErrorMemoryAllocation) an allocation that would
// exceed the budget set with mlens_set_device_memory_limit.
cudaError_t dmalloc_raw(void **p, size_t bytes);
void dfree(const void *p);
template <class T>
inline cudaError_t dmalloc(T **p, size_t bytes)
{
    return dmalloc_raw(reinterpret_cast<void **>(p), bytes);
}
BinGrid make_bin_grid(const mlens_grid &g);
RayGrid make_ray_grid(const mlens_grid &g);
LensTerms make_lens_terms(double kc, double g1, double g2);

}  // namespace mlens

struct FarState;                       // learned far field (farfield_api.cu)
void mlens_free_far_field(mlens_ctx *ctx);

// A star field on one device (definition shared by the API translation units).
struct mlens_ctx {
    int device = -1;
    int64_t n = 0;          // stars given
    int64_t n_pad = 0;      // stars on the device (multiple of kStarPad)
    float4 *d_stars = nullptr;
    unsigned long long *d_stats = nullptr;  // [binned, out, nan]
    mlens::LensTerms lens{};
    int precision = MLENS_PREC_FP32;
    int pairs_per_thread = 4;
    int star_stage = 256;
    int fma_pairs = mlens::kDefaultFmaPairs;
    int star_split = 0;     // 0 = automatic, else CTAs per tile (1 .. 8: clusters; above: through global memory)
    float4 *d_gpart = nullptr;  // the global split's partials (grown on demand)
    size_t gpart_bytes = 0;
    int nsm = 0;            // SMs of the context's device
    FarState *ff = nullptr;
};
