// shoot_fp32.cu -- the FP32 direct-sum ray-shooting kernels (Algorithm 1 with
// the deflection of Eq. 3 and the source position of Eq. 2), fused with the
// binning step.
//
// One CTA of 256 threads owns a 64 x (8*NP) tile of the ray grid; each thread
// owns 2*NP rays of one grid column, processed as NP packed pairs with the
// Blackwell f32x2 instructions (FADD2/FMUL2/FFMA2), so one instruction serves
// two rays.  Stars stream through shared memory in stages of 256; each stage
// is re-centred on the tile (star minus tile centre, once per star per CTA) and
// stored duplicated as (-dx,-dx,-dy,-dy),(m,m) so that a single broadcast
// LDS.128 + LDS.64 feeds every packed pair.  Per star and ray the work is
// FADD, FFMA (r^2), MUFU.RCP, FMUL (m/r^2), 2 FFMA (accumulate): the MUFU
// reciprocal (16 per SM per clock) is the only unit near saturation.
//
// Precision (MLENS_PREC_FP32): rays and stars are relative to an FP32 tile
// centre c, so differences of nearby positions are exact and the summed terms
// carry no absolute-coordinate rounding.  Terms are accumulated in plain FP32
// over 32 stars and each 32-star partial is added to the running sum with
// Kahan compensation.  The smooth+shear part A c of the tile centre is formed
// in FP64 once per tile, and beta = A c + A delta - S is assembled as a float
// pair, so the only rounding left at the full coordinate scale is the exact
// binning rule's.  MLENS_PREC_FP32_NAIVE keeps absolute coordinates and one
// running FP32 sum (Algorithm 1 written in single precision).
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_dev.cuh"

namespace mlens {

constexpr int kThreads = 256;
constexpr int kTileX = 64;                 // rays per tile row = threads per row group
constexpr int kGroups = kThreads / kTileX; // row groups
constexpr int kStage = 256;                // stars per shared-memory stage (one per thread)
constexpr int kKahan = 32;                 // stars per compensated partial

static_assert(kStage == kThreads, "one star per thread per stage");
static_assert(kStage % kKahan == 0, "stage must hold whole Kahan chunks");
static_assert(kStarPad % kStage == 0, "star padding must be whole stages");

struct StarStage {
    float4 q[2][kStage];   // (-dx, -dx, -dy, -dy) relative to the tile centre
    float2 mm[2][kStage];  // (m, m)
};

union ShootSmem {
    StarStage st;
    uint32_t hist[kWin * kWin];
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// v - c for packed pairs, with one rounding (fma with -1 is exact in the product)
__device__ __forceinline__ float2 sub2(float2 v, float2 c) { return __ffma2_rn(c, f2(-1.0f, -1.0f), v); }

// Kahan step on packed pairs: S + v with compensation C (true sum ~ S - C).
__device__ __forceinline__ void kahan2(float2 &S, float2 &C, float2 v)
{
    float2 y = sub2(v, C);
    float2 t = __fadd2_rn(S, y);
    C = sub2(sub2(t, S), y);
    S = t;
}

template <int NP, bool NAIVE>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_fp32(ShootArgs a)
{
    constexpr int kTileY = kGroups * 2 * NP;
    __shared__ __align__(16) ShootSmem sm;
    __shared__ float tc[8];        // cx, cy, ex, ey, B0h.x, B0h.y, B0l.x, B0l.y
    __shared__ int win[2];
    __shared__ unsigned sred[3];

    const int tid = threadIdx.x;
    const int tx = tid % kTileX;
    const int tg = tid / kTileX;
    const int i0 = blockIdx.x * kTileX;
    const int j0 = blockIdx.y * kTileY;
    const RayGrid &R = a.rays;

    if (tid == 0) {
        if (!NAIVE) {
            // tile centre (any float near the middle), offsets of the first ray and
            // A c in FP64, split into float pairs
            double cxd = R.x0 + ((double)i0 + 0.5 * kTileX) * R.dx;
            double cyd = R.y0 + ((double)j0 + 0.5 * kTileY) * R.dy;
            float cx = (float)cxd, cy = (float)cyd;
            double ex = (R.x0 + ((double)i0 + 0.5) * R.dx) - (double)cx;
            double ey = (R.y0 + ((double)j0 + 0.5) * R.dy) - (double)cy;
            double bx = a.lens.a11 * (double)cx + a.lens.a12 * (double)cy;
            double by = a.lens.a12 * (double)cx + a.lens.a22 * (double)cy;
            float bxh = (float)bx, byh = (float)by;
            tc[0] = cx;
            tc[1] = cy;
            tc[2] = (float)ex;
            tc[3] = (float)ey;
            tc[4] = bxh;
            tc[5] = byh;
            tc[6] = (float)(bx - (double)bxh);
            tc[7] = (float)(by - (double)byh);
        }
        sred[0] = sred[1] = sred[2] = 0u;
    }
    __syncthreads();

    // ------------------------------------------------------- this thread's rays
    float2 rx;       // packed (x, x): both rays of a pair share the column
    float2 ry[NP];   // packed (y_2p, y_2p+1)
    float2 px[NP], py[NP];             // partial sums (NAIVE: the whole running sum)
    float2 Sx[NP], Sy[NP], Cx[NP], Cy[NP];
    const float kx = (float)tx;
    float cx = 0.f, cy = 0.f;
    if (!NAIVE) {
        cx = tc[0];
        cy = tc[1];
        float dxr = __fmaf_rn(kx, R.dxh, __fmaf_rn(kx, R.dxl, tc[2]));
        rx = f2(dxr, dxr);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
            ry[p] = f2(__fmaf_rn(k0, R.dyh, __fmaf_rn(k0, R.dyl, tc[3])),
                       __fmaf_rn(k1, R.dyh, __fmaf_rn(k1, R.dyl, tc[3])));
            px[p] = py[p] = Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
        }
    } else {
        const float x0f = (float)R.x0, y0f = (float)R.y0;
        const float dxf = (float)R.dx, dyf = (float)R.dy;
        float thx = x0f + ((float)(i0 + tx) + 0.5f) * dxf;
        rx = f2(thx, thx);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float y0 = y0f + ((float)(j0 + tg * 2 * NP + 2 * p) + 0.5f) * dyf;
            float y1 = y0f + ((float)(j0 + tg * 2 * NP + 2 * p + 1) + 0.5f) * dyf;
            ry[p] = f2(y0, y1);
            // alpha_0 first (Algorithm 1), then every star is added to it
            px[p] = f2(a.lens.fm11 * thx + a.lens.fm12 * y0, a.lens.fm11 * thx + a.lens.fm12 * y1);
            py[p] = f2(a.lens.fm12 * thx + a.lens.fm22 * y0, a.lens.fm12 * thx + a.lens.fm22 * y1);
        }
    }

    // ---------------------------------------------------------- star stages
    const int nstage = (int)(a.nstars / kStage);
    auto stage_store = [&](int buf, float4 q) {
        float nx = NAIVE ? -q.x : __fsub_rn(cx, q.x);
        float ny = NAIVE ? -q.y : __fsub_rn(cy, q.y);
        sm.st.q[buf][tid] = make_float4(nx, nx, ny, ny);
        sm.st.mm[buf][tid] = f2(q.z, q.z);
    };
    if (nstage > 0) stage_store(0, __ldg(&a.stars[tid]));
    __syncthreads();

    for (int s = 0; s < nstage; ++s) {
        const int buf = s & 1;
        float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s + 1 < nstage) nxt = __ldg(&a.stars[(int64_t)(s + 1) * kStage + tid]);
        const float4 *Q = sm.st.q[buf];
        const float2 *M = sm.st.mm[buf];
#pragma unroll 1
        for (int k0 = 0; k0 < kStage; k0 += kKahan) {
#pragma unroll
            for (int k = k0; k < k0 + kKahan; ++k) {
                const float4 q = Q[k];
                const float2 m2 = M[k];
                const float2 dx = __fadd2_rn(rx, f2(q.x, q.y));
                const float2 dx2 = __fmul2_rn(dx, dx);
                const float2 nyv = f2(q.z, q.w);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float2 dy = __fadd2_rn(ry[p], nyv);
                    const float2 r2 = __ffma2_rn(dy, dy, dx2);
                    const float2 inv = f2(rcp_approx(r2.x), rcp_approx(r2.y));
                    const float2 f = __fmul2_rn(m2, inv);
                    px[p] = __ffma2_rn(f, dx, px[p]);
                    py[p] = __ffma2_rn(f, dy, py[p]);
                }
            }
            if (!NAIVE) {
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    kahan2(Sx[p], Cx[p], px[p]);
                    kahan2(Sy[p], Cy[p], py[p]);
                    px[p] = py[p] = f2(0.f, 0.f);
                }
            }
        }
        if (s + 1 < nstage) stage_store(buf ^ 1, nxt);
        __syncthreads();
    }

    // ------------------------------------------------ beta as float pairs
    float bxh[2 * NP], byh[2 * NP], bxl[2 * NP], byl[2 * NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 2 * p + h;
            if (!NAIVE) {
                const float sx = h ? Sx[p].y : Sx[p].x, sy = h ? Sy[p].y : Sy[p].x;
                const float ccx = h ? Cx[p].y : Cx[p].x, ccy = h ? Cy[p].y : Cy[p].x;
                const float dxr = rx.x, dyr = h ? ry[p].y : ry[p].x;
                // A delta for this ray (small)
                const float lx = __fmaf_rn(a.lens.fa11, dxr, __fmul_rn(a.lens.fa12, dyr));
                const float ly = __fmaf_rn(a.lens.fa12, dxr, __fmul_rn(a.lens.fa22, dyr));
                float th, tl;
                two_sum(tc[4], -sx, th, tl);
                tl = __fadd_rn(tl, __fadd_rn(__fadd_rn(tc[6], ccx), lx));
                two_sum(th, tl, bxh[r], bxl[r]);
                two_sum(tc[5], -sy, th, tl);
                tl = __fadd_rn(tl, __fadd_rn(__fadd_rn(tc[7], ccy), ly));
                two_sum(th, tl, byh[r], byl[r]);
            } else {
                const float thy = h ? ry[p].y : ry[p].x;
                bxh[r] = __fsub_rn(rx.x, h ? px[p].y : px[p].x);
                byh[r] = __fsub_rn(thy, h ? py[p].y : py[p].x);
                bxl[r] = 0.0f;
                byl[r] = 0.0f;
            }
        }
    }

    // ----------------------------------------------------------- binning
    const int ix = i0 + tx;
    const bool col_ok = ix < R.nx;
    __syncthreads();  // star stages are dead: reuse the memory as the window
    for (int b = tid; b < kWin * kWin; b += kThreads) sm.hist[b] = 0u;
    if (tid == 0) {
        win[0] = pair_axis_rough(bxh[0], a.bin.ax) - kWin / 2;
        win[1] = pair_axis_rough(byh[0], a.bin.ay) - kWin / 2;
    }
    __syncthreads();
    WinHist W{sm.hist, win[0], win[1]};
    unsigned nb = 0, no = 0, nn = 0;
#pragma unroll
    for (int r = 0; r < 2 * NP; ++r) {
        const int jy = j0 + tg * 2 * NP + r;
        uint32_t key = kNoKey;
        if (col_ok && jy < R.ny) {
            int gpx = 0, gpy = 0;
            const int pix = pair_pixel(bxh[r], byh[r], bxl[r], byl[r], a.bin, gpx, gpy);
            if (pix >= 0) {
                ++nb;
                key = hist_key(pix, gpx, gpy, W, a.bin);
            } else if (pix == -1) {
                ++no;
            } else {
                ++nn;
            }
            if (a.beta_out) {
                float4 *bo = reinterpret_cast<float4 *>(a.beta_out);
                bo[(int64_t)jy * R.nx + ix] = make_float4(bxh[r], byh[r], bxl[r], byl[r]);
            }
        }
        hist_add_warp(key, W, a.counts);
    }
    __syncthreads();
    hist_flush(W, a.bin, a.counts);
    stats_add_block(nb, no, nn, sred, a.stats);
}

template <int NP, bool NAIVE>
static cudaError_t launch_t(const ShootArgs &a, cudaStream_t s)
{
    constexpr int kTileY = kGroups * 2 * NP;
    dim3 grid((unsigned)((a.rays.nx + kTileX - 1) / kTileX), (unsigned)((a.rays.ny + kTileY - 1) / kTileY));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    k_shoot_fp32<NP, NAIVE><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_shoot_fp32(const ShootArgs &a, int pairs_per_thread, bool naive, cudaStream_t s)
{
    if (naive) return pairs_per_thread == 2 ? launch_t<2, true>(a, s) : launch_t<4, true>(a, s);
    return pairs_per_thread == 2 ? launch_t<2, false>(a, s) : launch_t<4, false>(a, s);
}

}  // namespace mlens
