// mlens_dev.cuh -- device helpers shared by the libmlens kernels:
// float-pair arithmetic, the exact float-pair binning rule (the source-pixel
// conversion of Algorithm 1) and the privatised, warp-aggregated histogram
// epilogue that performs its "mag[j_s, i_s] += 1".
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_internal.h"

namespace mlens {

// ------------------------------------------------------------ float pairs
// Knuth's error-free TwoSum: s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    float x = __fadd_rn(a, b);
    float bb = __fsub_rn(x, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(x, bb)), __fsub_rn(b, bb));
    s = x;
}

// MUFU reciprocal (max error 1 ulp; 1/0 = +inf).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------- exact binning rule
// Pixel of one axis for beta = bh + bl (an unevaluated float pair):
// floor((bh + bl - x0) * s) with x0 = x0h + x0l, s = sh + sl, evaluated as
// float pairs and floored exactly; -1 when outside [0, n).  The operation
// sequence is part of the library's contract (a CPU re-binning with the same
// float32 operations reproduces the GPU map bit for bit).
__device__ __forceinline__ int pair_axis_exact(float bh, float bl, const AxisPair &A)
{
    float dh, dl;
    two_sum(bh, -A.x0h, dh, dl);
    float t = __fsub_rn(bl, A.x0l);
    dl = __fadd_rn(dl, t);
    two_sum(dh, dl, dh, dl);
    float uh = __fmul_rn(dh, A.sh);
    float ul = __fmaf_rn(dh, A.sh, -uh);
    ul = __fmaf_rn(dh, A.sl, ul);
    ul = __fmaf_rn(dl, A.sh, ul);
    two_sum(uh, ul, uh, ul);
    if (!(uh == uh) || isinf(uh)) return -1;
    float p = floorf(uh);
    if (p == uh && ul < 0.0f) p = __fsub_rn(p, 1.0f);
    if (p < 0.0f || p >= (float)A.n) return -1;
    return (int)p;
}

// The same pixel, usually without the pair arithmetic.  u = fl(fl(bh - x0h) sh)
// differs from the pair value P = uh + ul that pair_axis_exact floors by at most
//     B = 2^-23 |u| (two roundings) + |d sl| + (|bl| + |x0l|)(|sh| + |sl|)
//         + 2^-23 (|bl| + |x0l|) |s| + 2^-45 |u| (the pair's own error),
// d = bh - x0h.  Since |sl| <= 2^-24 |sh| (sl is the rounding error of sh) and
// |d sh| <= (1 + 2^-23) |u|, the second term is at most 2^-24 (1 + 2^-23) |u|, so
//     B < 2^-22 |u| + (1 + 2^-22) (|bl| + |x0l|) |sh|.
// The quick test widens u by del = 2^-21 |u| + 2 |bl| |sh| + tq, with tq =
// 2 |x0l| |sh| + 2^-100 rounded up (so del > 0 where the products underflow):
// about twice B, which leaves room for del's own two roundings and those of
// u -/+ del (each under 2^-23 |u| + 2^-23 del).  If no pixel edge lies in
// [u - del, u + del], floor(P) = floor(u) and the result equals
// pair_axis_exact's bit for bit; otherwise (a fraction ~ 2 del of the rays, and
// every non-finite component: u or del is then inf or NaN) the exact rule runs.
//
// The quick decision alone: true, with p = pixel or -1 (outside [0, n)), when
// no pixel edge lies within del of u; false when the exact rule must run.
__device__ __forceinline__ bool pair_axis_quick(float bh, float bl, const AxisPair &A, int &p)
{
    const float d = __fsub_rn(bh, A.x0h);
    const float u = __fmul_rn(d, A.sh);
    const float del = __fmaf_rn(fabsf(u), 0x1p-21f, __fmaf_rn(fabsf(bl), A.sh2, A.tq));
    // floor(u + del) == lo  <=>  u + del < lo + 1 (u + del >= lo; where lo + 1
    // rounds to lo the test fails and the exact rule decides; NaN fails too)
    const float lo = floorf(__fsub_rn(u, del));
    if (!(__fadd_rn(u, del) < __fadd_rn(lo, 1.0f))) return false;
    p = (lo < 0.0f || lo >= (float)A.n) ? -1 : (int)lo;
    return true;
}

__device__ __forceinline__ int pair_axis(float bh, float bl, const AxisPair &A)
{
    int p;
    if (pair_axis_quick(bh, bl, A, p)) return p;
    return pair_axis_exact(bh, bl, A);
}

// Unclamped floor of the hi part (used only to place the histogram window).
__device__ __forceinline__ int pair_axis_rough(float bh, const AxisPair &A)
{
    float u = (bh - A.x0h) * A.sh;
    u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
    return (int)floorf(u);
}

// Classify one float-pair beta: returns linear pixel j*nx + i, -1 (out), -2 (non-finite).
__device__ __forceinline__ int pair_pixel(float xh, float yh, float xl, float yl, const BinGrid &g, int &px,
                                          int &py)
{
    if (!isfinite(xh) || !isfinite(yh) || !isfinite(xl) || !isfinite(yl)) return -2;
    px = pair_axis(xh, xl, g.ax);
    py = pair_axis(yh, yl, g.ay);
    if (px < 0 || py < 0) return -1;
    return py * g.nx + px;
}

// ------------------------------------------------ privatised histogram epilogue
// A CTA's rays come from one compact tile of the lens plane, so almost all of
// them land in a small patch of the source map.  The CTA counts that patch in
// a W x W shared-memory window (placed on the pixel of one of its rays), merges
// equal pixels across a warp with __match_any_sync before touching memory, and
// adds the window to the global map at the end; rays outside the window go
// straight to global atomics.
constexpr int kWin = 64;
constexpr uint32_t kNoKey = 0xffffffffu;

struct WinHist {
    uint32_t *h;   // kWin*kWin counters in shared memory
    int wx0, wy0;  // window origin in pixels
};

// key: < kWin*kWin for the window, kWin*kWin + pixel for a global pixel, kNoKey for none.
__device__ __forceinline__ uint32_t hist_key(int pix, int px, int py, const WinHist &W, const BinGrid &g)
{
    if (pix < 0) return kNoKey;
    int wx = px - W.wx0, wy = py - W.wy0;
    if ((unsigned)wx < (unsigned)kWin && (unsigned)wy < (unsigned)kWin) return (uint32_t)(wy * kWin + wx);
    return (uint32_t)(kWin * kWin) + (uint32_t)pix;
}

// Clear the window (uint4 stores; the window is 16-byte aligned).
__device__ __forceinline__ void hist_zero(uint32_t *h)
{
    uint4 *h4 = reinterpret_cast<uint4 *>(h);
    for (int b = threadIdx.x; b < kWin * kWin / 4; b += blockDim.x) h4[b] = make_uint4(0u, 0u, 0u, 0u);
}

// Warp-cooperative increment: every lane of the warp must call this together.
// Lanes hold neighbouring rays, whose pixels repeat in runs: the first lane of
// each run of equal keys adds the run's length (one atomic per run instead of
// one per ray; cheaper than matching all equal keys of the warp).
__device__ __forceinline__ void hist_add_warp(uint32_t key, const WinHist &W, uint32_t *counts)
{
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const bool start = lane == 0u || prev != key;
    const unsigned starts = __ballot_sync(0xffffffffu, start);
    if (start && key != kNoKey) {
        const unsigned later = starts & (0xfffffffeu << lane);
        const unsigned c = (later ? (unsigned)(__ffs(later) - 1) : 32u) - lane;
        if (key < (uint32_t)(kWin * kWin))
            atomicAdd(&W.h[key], c);
        else
            atomicAdd(&counts[key - (uint32_t)(kWin * kWin)], c);
    }
}

// Add the window to the global map (bins outside the map are never filled).
__device__ __forceinline__ void hist_flush(const WinHist &W, const BinGrid &g, uint32_t *counts)
{
    const uint4 *h4 = reinterpret_cast<const uint4 *>(W.h);
    for (int b = threadIdx.x; b < kWin * kWin / 4; b += blockDim.x) {
        const uint4 v = h4[b];
        if ((v.x | v.y | v.z | v.w) == 0u) continue;
        const int64_t base = (int64_t)(W.wy0 + b / (kWin / 4)) * g.nx + (W.wx0 + 4 * (b % (kWin / 4)));
        if (v.x) atomicAdd(&counts[base + 0], v.x);
        if (v.y) atomicAdd(&counts[base + 1], v.y);
        if (v.z) atomicAdd(&counts[base + 2], v.z);
        if (v.w) atomicAdd(&counts[base + 3], v.w);
    }
}

// Block-wide sum of three per-thread counters into global 64-bit stats.
__device__ __forceinline__ void stats_add_block(unsigned binned, unsigned out, unsigned nan, unsigned *sred,
                                                unsigned long long *stats)
{
    binned = __reduce_add_sync(0xffffffffu, binned);
    out = __reduce_add_sync(0xffffffffu, out);
    nan = __reduce_add_sync(0xffffffffu, nan);
    if ((threadIdx.x & 31u) == 0) {
        if (binned) atomicAdd(&sred[0], binned);
        if (out) atomicAdd(&sred[1], out);
        if (nan) atomicAdd(&sred[2], nan);
    }
    __syncthreads();
    if (threadIdx.x == 0 && stats) {
        if (sred[0]) atomicAdd(&stats[0], (unsigned long long)sred[0]);
        if (sred[1]) atomicAdd(&stats[1], (unsigned long long)sred[1]);
        if (sred[2]) atomicAdd(&stats[2], (unsigned long long)sred[2]);
    }
}

}  // namespace mlens
