// farfield.h -- structures of the learned-far-field variant shared by its
// kernels (farfield.cu) and its host API (farfield_api.cu).
//
// The lens plane around the ray grid is cut into square cells aligned with the
// 64 x 32-ray tiles of the FP32 kernels (a cell is ktx x kty tiles), plus one
// ring of cells around them so that every ray cell has its full 3 x 3 block.
// For a ray in cell c the stars of the 3 x 3 block are summed exactly (the near
// field); every other star contributes through the cell's far field
//     F(z) = sum_far m_k / (z - z_k),   alpha_far = conj(F),
// holomorphic on the block and expanded about the cell centre z_c in the series
// variable v = (z - z_c) / s, s = half the cell diagonal:
//     F = sum_p b_p v^p,   b_p = -sum_far m_k s^p / (z_k - z_c)^(p+1).
// Orders 0..Pe are evaluated exactly (b_0 as a float pair).  The remainder is
// v^(Pe+1) q(v) with q(v) = sum_{Pe < p <= Pt} b_p v^(p-Pe-1); the network
// learns q -- a slowly varying function dominated by b_(Pe+1) -- in units of
// the cell's bound s_c = sum_{Pe < p <= Pt} |b_p| (|q| <= s_c for |v| <= 1), and
// enters the series as its next coefficient.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_internal.h"

namespace mlens {

constexpr int kPtMax = 24;  // highest expansion order kept (targets)
constexpr int kPeMax = 16;  // highest order evaluated exactly
constexpr int kCoefStride = 4 + 2 * kPeMax;  // b0 hi/lo (re, im) + b1..bPe (re, im)

struct CellGrid {
    double x0, y0, w;  // origin and width of the extended grid (ray cells + 1 ring)
    int nx, ny;        // extended grid size
    int ncx, ncy;      // ray cells
    int ktx, kty;      // 64 x 32-ray tiles per cell
    int rays_nx, rays_ny;
};

__host__ __device__ inline int ext_index(const CellGrid &g, int cx, int cy) { return (cy + 1) * g.nx + (cx + 1); }

// The network constants every learned tile shares, per pair of hidden units
// (c, c + 1), c = 2 P, in the order the kernel's packed FP32 operations take them.
// Passed by value with the launch, so the kernel reads them from its constant bank
// instead of shared memory.  The constants of a pre-activation are halved (exact):
// the kernel forms SiLU's argument v / 2 directly.
constexpr int kNetPairs = 32;  // hidden units / 2
struct NetConsts {
    float4 w1u[kNetPairs];  // {W1u[c][0], W1u[c+1][0], W1u[c][1], W1u[c+1][1]} / 2
    float4 l2p[kNetPairs];  // {b2[c] / 2, b2[c+1] / 2, W3[0][c], W3[0][c+1]}
    float2 l2q[kNetPairs];  // {W3[1][c], W3[1][c+1]}
    float b3[2];
};

// Everything the learned shooting kernel reads.
struct LearnedArgs {
    ShootArgs plain;           // all stars, grids, counts, counters: used by fallback tiles and the epilogue
    CellGrid cg;
    const int *cstart;         // extended cells + 1: CSR offsets into cstars
    const float4 *cstars;      // stars sorted by extended cell (input order within a cell)
    const float *coef;         // per ray cell kCoefStride floats
    const float *sc;           // per ray cell residual bound s_c
    const int *flags;          // per ray cell: 1 = fall back to the plain sum
    const float *ec;           // per ray cell 64 floats: bf16(W1z) bf16(z_c) + b1
    const float *params;       // FP32 network parameters (flat layout of mlp.cuh)
    const __nv_bfloat16 *w2b;  // W2 in BF16, [out][in]
    int pe;
    int use_net;
    const int *items;          // tile index per work item (fallback tiles first)
    int64_t nitems;
    unsigned long long *counter;
    int *err;                  // set to 1 if a tensor-core completion wait gave up (results invalid)
    int wait_probe;            // test aid: each warpgroup's first wait polls an mbarrier nothing arrives on
    NetConsts net;             // the network's shared constants (use_net)
};

// Sample generation for training / validation (counter-based, SplitMix64).
struct SampleSpec {
    uint64_t seed;
    int64_t offset;      // index of the first sample of this launch
    int64_t count;       // samples in this launch
    int nrc;             // ray cells
    int per_cell;        // samples are dealt round-robin over cells: cell = index % nrc
};

struct TrainArgs {
    // network
    float *params;                     // FP32 master (read)
    const __nv_bfloat16 *w1zb, *w2b;   // BF16 copies of W1z [64][32] and W2 [64][64]
    const unsigned char *wimg;         // the same as the training kernel's shared-memory operands (16-byte aligned)
    float *grads;                      // host-side bookkeeping: the reduced gradients (flat layout)
    float *loss;                       // validation / forward-only: accumulated loss (sum of squared errors / B)
    // backward: each CTA writes its weight gradients and loss to row blockIdx.x of
    // gpart (ff_gpart_stride floats per row) and each sample its latent gradient
    // to dzs[sample][32]; ff_step_update (training) or ff_reduce_grads sums them in
    // a fixed order (deterministic training)
    float *gpart;
    float *dzs;
    // generated samples (training / validation)
    const float *z;                    // latents [nrc][32]
    float *dz;                         // latent gradients [nrc][32]
    const float *tail;                 // [nrc][2 (Pt - Pe)]
    const float *sc;                   // [nrc]
    CellGrid cg;
    int pe, pt;
    SampleSpec spec;
    float inv_batch;                   // 1 / B for the loss normalisation
    // explicit samples (verification): if zin != nullptr these are used instead
    const float *zin, *uin, *tin;      // [B][32], [B][2], [B][2]
    float *yout;                       // [B][2] network outputs (nullable)
    float *dzout;                      // [B][32] latent gradients (nullable)
    // validation outputs (forward only): per-cell max errors as float bits, sums
    unsigned *val_max_net, *val_max_series;
    double *val_sum;                   // [2]: sum of errors (network, series)
    int backward;                      // 0 = forward only (validation)
    int *err;                          // set to 1 if a tensor-core completion wait gave up (nullable)
    int wait_probe;                    // test aid: the CTA's first wait polls an mbarrier nothing arrives on
};

// launchers (farfield.cu)
cudaError_t ff_build_csr(const float4 *stars, int64_t n, const CellGrid &cg, int *scell, int *count, int *start,
                         int *fill, int *perm, float4 *cstars, cudaStream_t s);
cudaError_t ff_coefficients(const float4 *stars, const int *scell, int64_t n, const CellGrid &cg, int pt,
                            double *coef64, cudaStream_t s);
cudaError_t ff_convert(const double *coef64, const CellGrid &cg, int pe, int pt, float *coef, float *tail, float *sc,
                       cudaStream_t s);
cudaError_t ff_init_params(float *params, float *z, int nrc, uint64_t seed, cudaStream_t s);
// BF16 copies of W1z and W2, and the training kernel's image of its weight
// operands (ff_weight_image_bytes bytes, 16-byte aligned)
cudaError_t ff_prep_bf16(const float *params, __nv_bfloat16 *w1zb, __nv_bfloat16 *w2b, unsigned char *wimg,
                         cudaStream_t s);
int64_t ff_weight_image_bytes();
// pdl: launched with programmatic stream serialisation (the training loop: the
// sample generation overlaps the previous kernel's end)
cudaError_t ff_train_step(const TrainArgs &t, int64_t nsamples, cudaStream_t s, bool pdl = false);
// The rest of one training step in one launch: the fixed-order sums of the step's
// weight and latent gradients, then the Adam update.
struct StepUpdate {
    float *p, *m, *v;                  // parameters (weights, then latents), Adam moments
    const float *gpart;                // the step's CTA gradient rows
    int64_t nblk;                      // rows
    const float *dzs;                  // the step's per-sample latent gradients
    int64_t count, offset;             // samples of the step and the first one's index
    int nrc;                           // cells (latents)
    float *loss;                       // receives the step's loss (nullable)
    float lr_w, lr_z, b1, b2, eps, bc1, bc2;
    __nv_bfloat16 *w1zb, *w2b;         // BF16 copies of W1z and W2, refreshed
    unsigned char *wimg;               // and the training kernel's operand image
};
cudaError_t ff_step_update(const StepUpdate &u, cudaStream_t s);
int64_t ff_gpart_stride();                 // floats per CTA row of gpart
int64_t ff_train_blocks(int64_t nsamples);  // CTAs of one ff_train_step
cudaError_t ff_reduce_grads(const float *gpart, int64_t nblk, float *grads, float *loss, cudaStream_t s);
cudaError_t ff_embed(const float *params, const float *z, int nrc, float *ec, cudaStream_t s);
cudaError_t ff_flags(const unsigned *maxerr, int nrc, float tol, int *flags, cudaStream_t s);
// fallback tiles use the plain tile function with the context's fma_pairs setting
cudaError_t ff_shoot_learned(const LearnedArgs &L, int grid, int fma_pairs, cudaStream_t s);
cudaError_t ff_learned_grid(int *grid);
// The learned kernel's NetConsts from the flat FP32 parameters (host copy).
void ff_net_consts(const float *params_host, NetConsts *out);

}  // namespace mlens
