// farfield.cu -- kernels of the learned-far-field variant (see farfield.h):
// cell CSR of the stars, local-expansion coefficients of the far field (direct
// sums over the far stars, FP64-accurate), network training / validation with
// every product on the fifth-generation tensor cores (tcgen05, BF16 operands,
// FP32 accumulators in tensor memory), and the persistent shooting kernel that
// evaluates near field + series + network per ray (the network's 64 x 64 layer on
// tcgen05) and falls back to the exact direct sum on flagged cells.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "farfield.h"
#include "umma.cuh"
#include "mlp.cuh"
#include "tile.cuh"

namespace mlens {

using namespace mlp;

// ============================================================== cell CSR
__device__ __forceinline__ int star_cell(float4 q, const CellGrid &g)
{
    const double fx = floor(__ddiv_rn(__dsub_rn((double)q.x, g.x0), g.w));
    const double fy = floor(__ddiv_rn(__dsub_rn((double)q.y, g.y0), g.w));
    if (!(fx >= 0.0 && fx < (double)g.nx && fy >= 0.0 && fy < (double)g.ny)) return -1;
    return (int)fy * g.nx + (int)fx;
}

__global__ void k_cells_count(const float4 *stars, int64_t n, CellGrid g, int *scell, int *count)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = star_cell(stars[k], g);
    scell[k] = c;
    if (c >= 0) atomicAdd(&count[c], 1);
}

// exclusive scan of count[0..nc) into start[0..nc] by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_scan(const int *count, int nc, int *start)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const int chunk = (nc + 1023) / 1024;
    const int b = min(nc, tid * chunk), e = min(nc, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = tid ? part[tid - 1] : 0;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == 1023) start[nc] = part[1023];
}

__global__ void k_cells_scatter(const int *scell, int64_t n, const int *start, int *fill, int *perm)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = scell[k];
    if (c >= 0) perm[start[c] + atomicAdd(&fill[c], 1)] = (int)k;
}

// stars of one cell back into input order (deterministic near-field sums)
__global__ void k_cells_sort(const int *start, int nc, int *perm)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int b = start[c], e = start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        const int v = perm[i];
        int j = i - 1;
        while (j >= b && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

__global__ void k_cells_gather(const float4 *stars, const int *perm, const int *start, int nc, float4 *cstars)
{
    const int total = start[nc];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        cstars[i] = stars[perm[i]];
}

cudaError_t ff_build_csr(const float4 *stars, int64_t n, const CellGrid &cg, int *scell, int *count, int *start,
                         int *fill, int *perm, float4 *cstars, cudaStream_t s)
{
    const int nc = cg.nx * cg.ny;
    cudaError_t e;
    if ((e = cudaMemsetAsync(count, 0, sizeof(int) * nc, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(fill, 0, sizeof(int) * nc, s)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (n > 0) k_cells_count<<<nb, 256, 0, s>>>(stars, n, cg, scell, count);
    k_scan<<<1, 1024, 0, s>>>(count, nc, start);
    if (n > 0) k_cells_scatter<<<nb, 256, 0, s>>>(scell, n, start, fill, perm);
    k_cells_sort<<<(nc + 255) / 256, 256, 0, s>>>(start, nc, perm);
    k_cells_gather<<<1024, 256, 0, s>>>(stars, perm, start, nc, cstars);
    return cudaGetLastError();
}

// ===================================================== series coefficients
// One warp per ray cell, eight cells per CTA sharing each staged chunk of stars.
// b_0 (the far field's value at the centre, ~30 theta_E, needed to ~1e-9) is
// formed per star in double-float arithmetic (below) and accumulated in
// double-float.  For p >= 1 the terms -(m/s) w^(p+1) are formed in FP32 (relative
// error ~p 6e-8 per term, far below what the series needs), summed per lane in
// FP32 over a stage and accumulated in double-float, so the sums keep ~48 bits while
// all the work runs on the FP32 pipe.
// Double-float arithmetic (an unevaluated pair of floats, ~48 significant bits) on
// the FP32 pipe: Knuth's TwoSum, the FMA form of Dekker's TwoProduct, and one
// Newton step for the reciprocal.  Used for the order-0 far-field term, which
// needs more than FP32 but not the FP64 pipe's scarce throughput.
struct DF {
    float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_norm(float a, float b)  // |b| small against a
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.h, b.h);
    return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.h, b.h), e = __fmaf_rn(a.h, b.h, -p);
    return df_norm(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}
__device__ __forceinline__ DF df_mulf(DF a, float b)
{
    const float p = __fmul_rn(a.h, b), e = __fmaf_rn(a.h, b, -p);
    return df_norm(p, __fmaf_rn(a.l, b, e));
}
// The order-0 term's steps, shortened for their operands:
// x^2 + y^2: the two high products' sum by TwoSum; their rounding errors (exact, by
// FMA) and the cross terms 2 x_h x_l, 2 y_h y_l go into the low part (x_l^2 and
// y_l^2, 2^-48 of the result, are left out).
__device__ __forceinline__ DF df_sq_sum(DF x, DF y)
{
    const float px = __fmul_rn(x.h, x.h), ex = __fmaf_rn(x.h, x.h, -px);
    const float py = __fmul_rn(y.h, y.h), ey = __fmaf_rn(y.h, y.h, -py);
    const DF s = df_two_sum(px, py);
    const float lx = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, ex), ly = __fmaf_rn(__fadd_rn(y.h, y.h), y.l, ey);
    return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(lx, ly)));
}
// 1 / a: the hardware reciprocal y (relative error ~2^-23) and one Newton step,
// y (1 + r) with r = 1 - a y; 1 - (a y)_h is exact (Sterbenz: (a y)_h is within
// 2^-22 of 1), so r costs two subtractions.  Relative error ~r^2 + 2^-46, below
// 2^-43.
__device__ __forceinline__ DF df_rcp(DF a)
{
    const float y = rcp_approx(a.h);
    const DF ay = df_mulf(a, y);
    const float r = __fsub_rn(__fsub_rn(1.0f, ay.h), ay.l);
    return df_norm(y, __fmul_rn(y, r));
}
// Compensated running sum of double-float terms: s.h collects the terms' high
// parts with TwoSum, s.l their low parts and the TwoSum errors (normalised with
// df_norm when read).
__device__ __forceinline__ void df_acc(DF &s, DF t)
{
    const DF u = df_two_sum(s.h, t.h);
    s = {u.h, __fadd_rn(s.l, __fadd_rn(u.l, t.l))};
}

__device__ __forceinline__ float2 f2c(float x, float y) { return make_float2(x, y); }

// Order-0 term of one far star in double-float: -m / (z_k - z_c) = (-tr, ti), with
// w = s / (z_k - z_c) in FP32 for the higher orders.
struct FarTerm {
    DF tr, ti;
    float wr, wi;
};
__device__ __forceinline__ FarTerm far_term(float4 q, float zxh, float zxl, float zyh, float zyl, float fscale)
{
    FarTerm t;
    const DF dx = df_add(df_two_sum(q.x, -zxh), {-zxl, 0.0f});
    const DF dy = df_add(df_two_sum(q.y, -zyh), {-zyl, 0.0f});
    const DF inv = df_rcp(df_sq_sum(dx, dy));
    const DF mi = df_mulf(inv, q.z);
    t.tr = df_mul(mi, dx);
    t.ti = df_mul(mi, dy);
    const float si_s = __fmul_rn(inv.h, fscale);
    t.wr = __fmul_rn(dx.h, si_s);
    t.wi = -__fmul_rn(dy.h, si_s);
    return t;
}

// Sums over the warp's lanes of the per-lane partials v[p] of orders p + 1 = 1 ..
// kPtMax, scattered so that lane q receives the sum of order q (lane 0 and lanes
// beyond kPtMax receive zero): a fold of 32 columns (orders 0 .. 31, the missing
// ones zero) in five halving steps, the lane's bit deciding which half it keeps.
// The order of the additions is fixed.
__device__ __forceinline__ float warp_scatter_orders(float (&v)[kPtMax])
{
    static_assert(kPtMax < 32, "orders fit in one warp");
    const int lane = threadIdx.x & 31;
    float c[16];
    {  // step 16: columns 0..15 against 16..31 (column q holds v[q - 1])
        const bool up = (lane & 16) != 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float lo = j == 0 ? 0.0f : v[j - 1];
            const float hi = j + 15 < kPtMax ? v[j + 15] : 0.0f;
            const float give = up ? lo : hi, keep = up ? hi : lo;
            c[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
        }
    }
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1) {
        const bool up = (lane & step) != 0;
#pragma unroll
        for (int j = 0; j < step; ++j) {
            const float give = up ? c[j] : c[j + step], keep = up ? c[j + step] : c[j];
            c[j] = keep + __shfl_xor_sync(0xffffffffu, give, step);
        }
    }
    return c[0];
}

// Two CTAs per SM.  While the stage sums were accumulated in FP64 a third CTA (80
// registers, with spills) hid more latency than the spills cost; with the FP32-pipe
// accumulation the kernel is bound by the FMA pipe and two CTAs without spills are
// faster (0.245 -> 0.232 s for 22016 cells x 1e6 stars).
__global__ void __launch_bounds__(256, 2) k_coeffs(const float4 *stars, const int *scell, int64_t n, CellGrid g, int pt,
                                                double scale, double *out)
{
    // One warp per ray cell.  Per far star: the order-0 term -m / (z_k - z_c) in
    // double-float arithmetic on the FP32 pipe, summed per lane over each stage's
    // stars and added to an FP64 accumulator once per stage; w = s / (z_k - z_c)
    // in FP32 and the higher orders t_p = t_0 w^p by an FP32 recurrence into
    // per-lane FP32 partials, summed across the warp after each 256-star stage,
    // lane p adding coefficient p's stage sum to its FP64 accumulator.  A lane
    // takes its stars in pairs (k, k + 32) and runs the two recurrences as packed
    // f32x2 operations (the pair's terms are added before they enter the partials,
    // which keeps the partials in 48 registers: two CTAs per SM).  Near stars, and the padding of a short stage, enter as a
    // massless star far away: they contribute exactly zero and keep the loop
    // uniform across the warp.
    __shared__ float4 sq[256];
    __shared__ int2 scl[256];  // the star's cell (x, y); (-8, -8) outside the grid
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrc = g.ncx * g.ncy;
    const int rc = blockIdx.x * 8 + warp;
    const bool ok = rc < nrc;
    const int ex = (ok ? rc % g.ncx : 0) + 1, ey = (ok ? rc / g.ncx : 0) + 1;
    const double zx = g.x0 + ((double)ex + 0.5) * g.w, zy = g.y0 + ((double)ey + 0.5) * g.w;
    // the cell centre as float pairs (48 bits of it; the star positions are floats)
    const float zxh = (float)zx, zxl = (float)(zx - (double)zxh);
    const float zyh = (float)zy, zyl = (float)(zy - (double)zyh);
    const float fscale = (float)scale;
    const float4 pad = make_float4(kPadCoord, kPadCoord, 0.0f, 0.0f);
    // running sums in double-float on the FP32 pipe (GB300's FP64 rate is a small
    // fraction of FP32: FP64 accumulation once per stage had made the FP64 pipe the
    // kernel's bound)
    DF b0r = {0.0f, 0.0f}, b0i = {0.0f, 0.0f};    // order 0, this lane's stars
    DF accr = {0.0f, 0.0f}, acci = {0.0f, 0.0f};  // lane p (1 <= p <= pt): coefficient p, all stages
    for (int64_t s0 = 0; s0 < n; s0 += 256) {
        const int cnt = (int)min((int64_t)256, n - s0);
        __syncthreads();
        {
            const int t = threadIdx.x;
            float4 q = pad;
            int2 cc = make_int2(-8, -8);
            if (t < cnt) {
                q = stars[s0 + t];
                const int c = scell[s0 + t];
                if (c >= 0) cc = make_int2(c % g.nx, c / g.nx);
            }
            sq[t] = q;
            scl[t] = cc;
        }
        __syncthreads();
        if (!ok) continue;
        float pr[kPtMax], pi[kPtMax];  // partial sums of order p + 1
#pragma unroll
        for (int p = 0; p < kPtMax; ++p) pr[p] = pi[p] = 0.0f;
        DF sr = {0.0f, 0.0f}, si = {0.0f, 0.0f};
        for (int j = 0; j < (cnt + 63) / 64; ++j) {
            const int ka = lane + 64 * j, kb = ka + 32;
            const int2 ca = scl[ka], cb = scl[kb];
            const bool near_a = abs(ca.x - ex) <= 1 && abs(ca.y - ey) <= 1;
            const bool near_b = abs(cb.x - ex) <= 1 && abs(cb.y - ey) <= 1;
            const FarTerm A = far_term(near_a ? pad : sq[ka], zxh, zxl, zyh, zyl, fscale);
            const FarTerm B = far_term(near_b ? pad : sq[kb], zxh, zxl, zyh, zyl, fscale);
            df_acc(sr, {-A.tr.h, -A.tr.l});
            df_acc(si, A.ti);
            df_acc(sr, {-B.tr.h, -B.tr.l});
            df_acc(si, B.ti);
            float2 fr = f2c(-A.tr.h, -B.tr.h), fi = f2c(A.ti.h, B.ti.h);
            const float2 wr = f2c(A.wr, B.wr), wi = f2c(A.wi, B.wi), nwi = f2c(-A.wi, -B.wi);
#pragma unroll
            for (int p = 0; p < kPtMax; ++p) {
                const float2 tr = __fmul2_rn(fr, wr), ti = __fmul2_rn(fr, wi);
                fr = __ffma2_rn(fi, nwi, tr);  // fr wr - fi wi
                fi = __ffma2_rn(fi, wr, ti);   // fr wi + fi wr
                pr[p] += __fadd_rn(fr.x, fr.y);
                pi[p] += __fadd_rn(fi.x, fi.y);
            }
        }
        b0r = df_add(b0r, df_norm(sr.h, sr.l));
        b0i = df_add(b0i, df_norm(si.h, si.l));
        // the stage's sums over the warp, scattered: afterwards lane q holds the sum of
        // order q (q = 1 .. kPtMax) of the stage (reduce-scatter, 31 shuffles per part)
        const float r = warp_scatter_orders(pr), i = warp_scatter_orders(pi);
        accr = df_add(accr, {r, 0.0f});
        acci = df_add(acci, {i, 0.0f});
    }
    if (!ok) return;
    double c0r = (double)b0r.h + (double)b0r.l, c0i = (double)b0i.h + (double)b0i.l;
    for (int o = 16; o; o >>= 1) {
        c0r += __shfl_xor_sync(0xffffffffu, c0r, o);
        c0i += __shfl_xor_sync(0xffffffffu, c0i, o);
    }
    double *dst = out + (int64_t)rc * (pt + 1) * 2;
    if (lane == 0) {
        dst[0] = c0r;
        dst[1] = c0i;
    } else if (lane <= pt) {
        dst[2 * lane] = (double)accr.h + (double)accr.l;
        dst[2 * lane + 1] = (double)acci.h + (double)acci.l;
    }
}

cudaError_t ff_coefficients(const float4 *stars, const int *scell, int64_t n, const CellGrid &cg, int pt,
                            double *coef64, cudaStream_t s)
{
    const int nrc = cg.ncx * cg.ncy;
    const double scale = cg.w * 0.70710678118654752440;
    k_coeffs<<<(nrc + 7) / 8, 256, 0, s>>>(stars, scell, n, cg, pt, scale, coef64);
    return cudaGetLastError();
}

__global__ void k_convert(const double *c64, int nrc, int pe, int pt, float *coef, float *tail, float *sc)
{
    const int rc = blockIdx.x * blockDim.x + threadIdx.x;
    if (rc >= nrc) return;
    const double *c = c64 + (int64_t)rc * (pt + 1) * 2;
    float *o = coef + (int64_t)rc * kCoefStride;
    const float rh = (float)c[0], ih = (float)c[1];
    o[0] = rh;
    o[1] = ih;
    o[2] = (float)(c[0] - (double)rh);
    o[3] = (float)(c[1] - (double)ih);
    for (int p = 1; p <= kPeMax; ++p) {
        o[4 + 2 * (p - 1)] = p <= pe ? (float)c[2 * p] : 0.0f;
        o[5 + 2 * (p - 1)] = p <= pe ? (float)c[2 * p + 1] : 0.0f;
    }
    double bound = 0.0;
    float *t = tail + (int64_t)rc * 2 * (pt - pe);
    for (int p = pe + 1; p <= pt; ++p) {
        t[2 * (p - pe - 1)] = (float)c[2 * p];
        t[2 * (p - pe - 1) + 1] = (float)c[2 * p + 1];
        bound += sqrt(c[2 * p] * c[2 * p] + c[2 * p + 1] * c[2 * p + 1]);
    }
    sc[rc] = (float)fmax(bound, 1e-30);
}

cudaError_t ff_convert(const double *coef64, const CellGrid &cg, int pe, int pt, float *coef, float *tail, float *sc,
                       cudaStream_t s)
{
    const int nrc = cg.ncx * cg.ncy;
    k_convert<<<(nrc + 255) / 256, 256, 0, s>>>(coef64, nrc, pe, pt, coef, tail, sc);
    return cudaGetLastError();
}

// ======================================================= network set-up
// SplitMix64 (Steele, Lea and Flood 2014): a counter-based 64-bit generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float unit24(uint64_t h) { return (float)(h >> 40) * (1.0f / 16777216.0f); }

__global__ void k_init_params(float *params, float *z, int nrc, uint64_t seed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nz = (int64_t)nrc * kLat;
    if (i < kParams) {
        float a = 0.0f;  // Glorot-uniform bound
        if (i < ob1) a = sqrtf(6.0f / (kLat + 2 + kHid));
        else if (i >= oW2 && i < ob2) a = sqrtf(6.0f / (2 * kHid));
        else if (i >= oW3 && i < ob3) a = sqrtf(6.0f / (kHid + kOut));
        params[i] = a * (2.0f * unit24(splitmix64(seed * 0x100000001B3ull + (uint64_t)i)) - 1.0f);
    } else if (i < kParams + nz) {
        const int64_t j = i - kParams;
        z[j] = 0.01f * (2.0f * unit24(splitmix64(seed * 0x100000001B3ull + 0x5bd1e995ull + (uint64_t)j)) - 1.0f);
    }
}

cudaError_t ff_init_params(float *params, float *z, int nrc, uint64_t seed, cudaStream_t s)
{
    const int64_t n = kParams + (int64_t)nrc * kLat;
    k_init_params<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, z, nrc, seed);
    return cudaGetLastError();
}

// Programmatic dependent launch between the training steps' kernels: a kernel
// launched with programmatic stream serialisation may begin while the one before
// it finishes; pdl_wait() returns once that one has completed and its writes are
// visible, and pdl_launch_next() lets the next kernel begin launching once every
// CTA of this one has called it.  Both do nothing in a kernel launched without
// the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ===================================================== training kernel
constexpr int kWaitPolls = 1 << 20;  // bound on a tensor-core completion wait
constexpr int kProbePolls = 1024;    // bound on a probe wait (an mbarrier nothing arrives on)
constexpr int kSampC = 128;          // samples per chunk = tensor-memory lanes of one accumulator
constexpr int kChunks = 2;           // chunks per CTA, one after the other
constexpr int kSampCTA = kChunks * kSampC;
constexpr int kGP = kParams + 2;     // gpart row: the parameters' gradients, then the loss

// Shared memory of the training kernel (byte offsets).  Every tensor-core
// operand is a row-major BF16 block [R][C] of 8-row x 16-byte core matrices:
// element (r, c) at tc_off(r, c, C), 128 bytes between core matrices along a row
// and 16 C bytes between 8-row groups.  A product whose K runs along the rows
// (over the columns c) reads the block K-major; one whose K runs down the columns
// (over the rows r: the weight gradients' sums over samples, the backward
// products' sums over output units) reads the same block MN-major.  Every block is
// written once, in its natural row order, with 16-byte stores.
__host__ __device__ constexpr int tc_off(int r, int k, int K)
{
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
struct TrainTc {
    // the weights [out][in]: B operands K-major for the forward products, MN-major for
    // the backward ones (dA1 = dH2 W2, dZ = dH1 W1z)
    static constexpr int W1z = 0;                        // [64 out][32 in]  layer 1, latent block
    static constexpr int W2 = W1z + kHid * kLat * 2;     // [64 out][64 in]  layer 2
    // per-sample blocks [128 samples][units]: A operands K-major for the per-sample
    // products; MN-major, over their samples, for the weight gradients: dW2 = dH2^T A1
    // and dW1z = dH1^T Z from the stacked [dH2 | dH1] (M = 128 units) against A1 and Z
    static constexpr int Z = W2 + kHid * kHid * 2;       // [128][32]
    static constexpr int A1 = Z + kSampC * kLat * 2;     // [128][64]
    static constexpr int DH = A1 + kSampC * kHid * 2;    // [128][128]: dh2 in units 0..63, dh1 in 64..127
    static constexpr int EndOps = DH + kSampC * 2 * kHid * 2;
    // FP32 / int region
    static constexpr int W1u = EndOps;                   // [64][2]
    static constexpr int b1 = W1u + 2 * kHid * 4;
    static constexpr int b2 = b1 + kHid * 4;
    static constexpr int W3 = b2 + kHid * 4;             // [2][64]
    static constexpr int b3 = W3 + 2 * kHid * 4;         // [2], padded
    // the CTA's samples, both chunks (sample i of chunk c at index c * 128 + i)
    static constexpr int U = b3 + 16;                    // [256][2] positions
    static constexpr int T = U + 2 * kSampCTA * 4;       // [256][2] targets
    static constexpr int SV = T + 2 * kSampCTA * 4;      // [256] s_c |v|^(pe+1)
    static constexpr int RC = SV + kSampCTA * 4;         // [256] int cell
    static constexpr int OK = RC + kSampCTA * 4;         // [256] int valid
    static constexpr int YP = OK + kSampCTA * 4;         // [2 warpgroups][128][2] layer-3 partial sums
    static constexpr int Slots = YP + 2 * kSampC * 2 * 4;  // [8 warps][6][32] column sums over a warp's samples
    static constexpr int WS = Slots + 8 * 6 * 32 * 4;    // [8 warps][4]: sum dy0, sum dy1, loss
    static constexpr int bytes = WS + 8 * 4 * 4;
    // tensor-memory columns (all 128 lanes).  A chunk's own accumulators are reused
    // once read: H1 and H2 first; dA1 over H2 once the dh2 pass has read it; dZ over
    // dA1 once the dh1 pass has read it.  dW2 and dW1z have columns of their own:
    // both chunks accumulate into them.
    static constexpr int cH1 = 0, cH2 = 64, cDA1 = 64, cDZ = 64, cDW2 = 128, cDW1z = 192, ncols = 256;
};
// two CTAs per SM: their dynamic and static shared memory within the SM's 228 KB
// less 1 KB per CTA, and their tensor memory within the SM's 512 columns (tensor
// memory allows no more than two)
static_assert(TrainTc::bytes + 128 <= (228 * 1024) / 2 - 1024, "two training CTAs per SM");
static_assert(2 * TrainTc::ncols <= 512, "two training CTAs per SM");

// The training kernel's weight operands as they sit in its shared memory (W1z and
// W2 at their TrainTc offsets): written wherever the BF16 weight copies are
// refreshed, so that a training CTA stages them with 16-byte copies.
constexpr int kWImgBytes = TrainTc::Z;
static_assert(kWImgBytes % 16 == 0, "the weight image is copied in 16-byte units");

// Entry i of the flat parameter vector (a W1z or W2 weight), rounded to BF16, into
// its place in the image.
__device__ __forceinline__ void wimg_put(unsigned char *img, int64_t i, __nv_bfloat16 b)
{
    using L = TrainTc;
    if (i >= oW1z && i < oW1z + kHid * kLat) {
        const int o = (int)(i - oW1z) / kLat, k = (int)(i - oW1z) % kLat;
        *reinterpret_cast<__nv_bfloat16 *>(img + L::W1z + tc_off(o, k, kLat)) = b;
    } else if (i >= oW2 && i < oW2 + kHid * kHid) {
        const int o = (int)(i - oW2) / kHid, k = (int)(i - oW2) % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(img + L::W2 + tc_off(o, k, kHid)) = b;
    }
}

__global__ void k_prep_bf16(const float *p, __nv_bfloat16 *w1zb, __nv_bfloat16 *w2b, unsigned char *wimg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kHid) {
        const __nv_bfloat16 b = to_bf16(p[oW2 + i]);
        w2b[i] = b;
        wimg_put(wimg, oW2 + i, b);
    }
    if (i < kHid * kLat) {
        const __nv_bfloat16 b = to_bf16(p[oW1z + i]);
        w1zb[i] = b;
        wimg_put(wimg, oW1z + i, b);
    }
}

cudaError_t ff_prep_bf16(const float *params, __nv_bfloat16 *w1zb, __nv_bfloat16 *w2b, unsigned char *wimg,
                         cudaStream_t s)
{
    k_prep_bf16<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(params, w1zb, w2b, wimg);
    return cudaGetLastError();
}

int64_t ff_weight_image_bytes() { return kWImgBytes; }

// One training / validation sample: a cell and a uniform position in its ray-covered
// part; the target is q(v) / s_c with q(v) = sum_{pe < p <= pt} b_p v^(p-pe-1) (so that
// the series remainder is v^(pe+1) q(v)); vp = |v|^(pe+1) turns errors in q into
// errors of the far field.
__device__ __forceinline__ void sample_of(const TrainArgs &A, int64_t li, int &rc, float &ux, float &uy, float &tx,
                                          float &ty, float &scv, float &vp)
{
    const int64_t i = A.spec.offset + li;
    rc = (int)(i % A.spec.nrc);
    const uint64_t h1 = splitmix64(A.spec.seed + 2ull * (uint64_t)i);
    const uint64_t h2 = splitmix64(A.spec.seed + 2ull * (uint64_t)i + 1ull);
    const int cx = rc % A.cg.ncx, cy = rc / A.cg.ncx;
    const float covx = fminf(1.0f, (float)(A.cg.rays_nx - cx * 64 * A.cg.ktx) / (float)(64 * A.cg.ktx));
    const float covy = fminf(1.0f, (float)(A.cg.rays_ny - cy * 32 * A.cg.kty) / (float)(32 * A.cg.kty));
    ux = 2.0f * unit24(h1) * covx - 1.0f;
    uy = 2.0f * unit24(h2) * covy - 1.0f;
    // q(v) at v = u / sqrt(2) by Horner, the cell's coefficients loaded first (all
    // in flight together; the row is 8-byte aligned)
    const float vr = ux * 0.70710678f, vi = uy * 0.70710678f;
    const int nt = A.pt - A.pe;
    const float2 *b = reinterpret_cast<const float2 *>(A.tail + (int64_t)rc * 2 * nt);
    float2 bc[kPtMax];
#pragma unroll
    for (int i = 0; i < kPtMax; ++i) bc[i] = i < nt ? b[i] : make_float2(0.0f, 0.0f);
    float ar = 0.0f, ai = 0.0f;
#pragma unroll
    for (int i = kPtMax - 1; i >= 0; --i) {
        if (i >= nt) continue;
        const float nr = ar * vr - ai * vi + bc[i].x;
        const float ni = ar * vi + ai * vr + bc[i].y;
        ar = nr;
        ai = ni;
    }
    scv = A.sc[rc];
    tx = ar / scv;
    ty = ai / scv;
    vp = powf(vr * vr + vi * vi, 0.5f * (float)(A.pe + 1));
}

// Column sums of 16 per-lane values over the warp's 32 lanes: afterwards lanes j
// and j + 16 hold the sum of column j (a fold, then a reduce-scatter; fixed order,
// so deterministic).
__device__ __forceinline__ float warp_colsum16(float (&v)[16])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
#pragma unroll
    for (int step = 8; step >= 1; step >>= 1) {
        const bool up = (lane & step) != 0;
#pragma unroll
        for (int i = 0; i < step; ++i) {
            const float give = up ? v[i] : v[i + step];
            const float keep = up ? v[i + step] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, step);
        }
    }
    return v[0];
}

// Make this thread's shared-memory operand writes visible to the tensor cores and
// wait for the whole CTA.
__device__ __forceinline__ void tc_publish()
{
    umma::fence_async_smem();
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
}

// Wait (bounded) for the MMAs committed to *bar; true when every thread saw them
// complete.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t &phase, uint64_t *probe = nullptr)
{
    // probe (test aid): wait instead on an mbarrier nothing arrives on, so the
    // bounded wait runs out and the failure path is taken
    const bool ok = probe ? umma::mbar_wait(probe, 0, kProbePolls) : umma::mbar_wait(bar, phase, kWaitPolls);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1u;
    umma::fence_after();
    return true;
}

// 16 accumulator columns of this thread's lane.
__device__ __forceinline__ void tc_load16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    umma::ld16(taddr, r);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void st_f4x4(float *dst, const float (&v)[16])  // 16-byte aligned
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// An operand of a product: a block of tc_off core matrices with `cols` columns,
// starting at byte `off` of shared memory, read K-major (K along its columns) or
// MN-major (K down its rows).
struct TcOp {
    int off, cols;
    bool mn;
    // descriptor strides: along K, along M/N, and the advance per K = 16 step
    __device__ __forceinline__ uint32_t lbo() const { return mn ? (uint32_t)(cols * 16) : 128u; }
    __device__ __forceinline__ uint32_t sbo() const { return mn ? 128u : (uint32_t)(cols * 16); }
    __device__ __forceinline__ uint32_t step() const { return mn ? (uint32_t)(cols * 32) : 256u; }
};

// One thread issues D = sum_k A[:, k] B[:, k]^T over K / 16 MMAs of K = 16 (acc:
// D += instead); M = 128.
__device__ __forceinline__ void tc_gemm(uint32_t d, const unsigned char *S, TcOp A, TcOp B, int N, int K,
                                        bool acc = false)
{
    const uint32_t a = umma::smem_addr(S + A.off), b = umma::smem_addr(S + B.off);
    const uint32_t idesc = umma::idesc_bf16(128, N, A.mn, B.mn);
    for (int ks = 0; ks < K / 16; ++ks)
        umma::mma_bf16(d, umma::desc(a + ks * A.step(), A.lbo(), A.sbo()),
                       umma::desc(b + ks * B.step(), B.lbo(), B.sbo()), idesc, acc || ks > 0 ? 1u : 0u);
}

// 16 latent columns (16 wg .. 16 wg + 15) of sample li of the launch, zero past its
// end: explicit latents, or those of the sample's cell (offset + li) mod nrc.
__device__ __forceinline__ void load_latents(const TrainArgs &A, int64_t li, int wg, float (&zv)[16])
{
    const bool ok = li < A.spec.count;
    const float *src = A.zin ? A.zin + li * kLat : A.z + ((A.spec.offset + li) % A.spec.nrc) * kLat;
    src += 16 * wg;
    if (!ok) {
#pragma unroll
        for (int j = 0; j < 16; ++j) zv[j] = 0.0f;
    } else if (((uintptr_t)src & 7u) == 0) {  // the latents (after the 6530 parameters) are 8-byte aligned
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 v = reinterpret_cast<const float2 *>(src)[j];
            zv[2 * j] = v.x;
            zv[2 * j + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) zv[j] = src[j];
    }
}

// The step for chunk `chunk` of the CTA's samples (128 of them); false if a
// tensor-core wait gave up (the caller drains and reports).  Thread (warpgroup wg,
// s = tid % 128) owns sample s and, of each 64-wide accumulator, the columns
// 32 wg .. 32 wg + 31, taken in two halves of 16 (tensor-memory lane s is readable
// by warp s / 32 of either warpgroup).  H1 and H2 are read back from tensor memory
// when the backward pass needs them rather than held in registers: two CTAs fit
// per SM.  zv holds the chunk's latents on entry and, after a backward chunk
// followed by another, the next chunk's (loaded while the last MMAs run).  The
// weight gradients and FP32 column sums accumulate over the chunks; the last one
// writes the CTA's gradient row.
__device__ __forceinline__ bool train_step(const TrainArgs &A, unsigned char *S, uint64_t *bar, uint64_t *idle,
                                           uint32_t tm, uint32_t &phase, float (&zv)[16], int chunk)
{
    using L = TrainTc;
    float *F = reinterpret_cast<float *>(S);  // byte offsets / 4 below
    int *I = reinterpret_cast<int *>(S);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, wg = warp >> 2, s = tid & 127;
    const int c0 = 32 * wg;  // this thread's first column of a 64-wide accumulator
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int64_t cbase = (int64_t)blockIdx.x * kSampCTA + chunk * kSampC;
    const int si = chunk * kSampC + s;  // the sample's index in the CTA's sample regions
    const bool expl = A.zin != nullptr, first = chunk == 0, last = chunk == kChunks - 1;
    float *Slot = F + L::Slots / 4 + warp * 6 * 32;
    // this warp's column sums so far plus r (the first chunk starts them)
    auto slot_add = [&](int i, float r) { Slot[i] = first ? r : Slot[i] + r; };
    const float ux = F[L::U / 4 + 2 * si], uy = F[L::U / 4 + 2 * si + 1];
    // pre-activations of layer 1 / layer 2 for columns c .. c + 15, from tensor memory
    auto load_h1 = [&](int c, float (&h)[16]) {
        tc_load16(tm + lane_base + L::cH1 + c, h);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            h[j] = h[j] + F[L::W1u / 4 + 2 * (c + j)] * ux + F[L::W1u / 4 + 2 * (c + j) + 1] * uy + F[L::b1 / 4 + c + j];
    };
    auto load_h2 = [&](int c, float (&h)[16]) {
        tc_load16(tm + lane_base + L::cH2 + c, h);
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] += F[L::b2 / 4 + c + j];
    };

    // ---- latents (gathered at kernel start): thread (wg, s) has columns 16 wg .. 16 wg + 15 of z_s
    {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<uint4 *>(S + L::Z + tc_off(s, 16 * wg + 8 * h, kLat)) =
                make_uint4(pack_bf16(zv[8 * h], zv[8 * h + 1]), pack_bf16(zv[8 * h + 2], zv[8 * h + 3]),
                           pack_bf16(zv[8 * h + 4], zv[8 * h + 5]), pack_bf16(zv[8 * h + 6], zv[8 * h + 7]));
    }
    // ---- layer 1, latent block: H1 = Z W1z^T (M 128, N 64, K 32)
    tc_publish();
    if (tid == 0) {
        tc_gemm(tm + L::cH1, S, TcOp{L::Z, kLat, false}, TcOp{L::W1z, kLat, false}, kHid, kLat);
        umma::commit(bar);
    }
    if (!tc_wait(bar, phase, A.wait_probe && first ? idle : nullptr)) return false;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {  // A1 = silu(H1 + W1u u + b1)
        const int c = c0 + 16 * hh;
        float h1[16];
        load_h1(c, h1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = silu1(h1[8 * q + j]);
            *reinterpret_cast<uint4 *>(S + L::A1 + tc_off(s, c + 8 * q, kHid)) =
                make_uint4(pack_bf16(a[0], a[1]), pack_bf16(a[2], a[3]), pack_bf16(a[4], a[5]), pack_bf16(a[6], a[7]));
        }
    }
    // ---- layer 2: H2 = A1 W2^T (M 128, N 64, K 64); layer 3 in FP32
    tc_publish();
    if (tid == 0) {
        tc_gemm(tm + L::cH2, S, TcOp{L::A1, kHid, false}, TcOp{L::W2, kHid, false}, kHid, kHid);
        umma::commit(bar);
    }
    if (!tc_wait(bar, phase)) return false;
    {
        float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int c = c0 + 16 * hh;
            float h2[16];
            load_h2(c, h2);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float a2 = silu2(h2[j]);
                y0 += F[L::W3 / 4 + c + j] * a2;
                y1 += F[L::W3 / 4 + kHid + c + j] * a2;
            }
        }
        F[L::YP / 4 + (wg * kSampC + s) * 2] = y0;
        F[L::YP / 4 + (wg * kSampC + s) * 2 + 1] = y1;
    }
    __syncthreads();
    // ---- outputs, loss, validation (both warpgroups form the same y and dy)
    const bool valid = I[L::OK / 4 + si] != 0;
    const float yv0 = F[L::YP / 4 + 2 * s] + F[L::YP / 4 + (kSampC + s) * 2] + F[L::b3 / 4];
    const float yv1 = F[L::YP / 4 + 2 * s + 1] + F[L::YP / 4 + (kSampC + s) * 2 + 1] + F[L::b3 / 4 + 1];
    const float ex = yv0 - F[L::T / 4 + 2 * si], ey = yv1 - F[L::T / 4 + 2 * si + 1];
    const float dy0 = valid ? 2.0f * ex * A.inv_batch : 0.0f, dy1 = valid ? 2.0f * ey * A.inv_batch : 0.0f;
    float lsum = valid && wg == 0 ? ex * ex + ey * ey : 0.0f;
    if (valid && wg == 0) {
        if (A.yout) {
            A.yout[2 * (cbase + s)] = yv0;
            A.yout[2 * (cbase + s) + 1] = yv1;
        }
        if (!A.backward && A.val_max_net) {
            const float scv = F[L::SV / 4 + si];
            const float en = scv * sqrtf(ex * ex + ey * ey);
            const float tx = F[L::T / 4 + 2 * si], ty = F[L::T / 4 + 2 * si + 1];
            const float es = scv * sqrtf(tx * tx + ty * ty);
            const int rc = I[L::RC / 4 + si];
            atomicMax(&A.val_max_net[rc], __float_as_uint(en));
            atomicMax(&A.val_max_series[rc], __float_as_uint(es));
            atomicAdd(&A.val_sum[0], (double)en);
            atomicAdd(&A.val_sum[1], (double)es);
        }
    }
    for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (!A.backward) {
        if (lane == 0 && wg == 0 && A.loss) atomicAdd(A.loss, lsum * A.inv_batch);
        return true;
    }
    {
        float d0 = wg == 0 ? dy0 : 0.0f, d1 = wg == 0 ? dy1 : 0.0f;
        for (int o = 16; o; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        if (lane == 0) {
            float *ws = F + L::WS / 4 + warp * 4;
            ws[0] = first ? d0 : ws[0] + d0;
            ws[1] = first ? d1 : ws[1] + d1;
            ws[2] = first ? lsum : ws[2] + lsum;
        }
    }
    // ---- dh2 = (dy W3) silu'(h2) into units 0..63 of DH; FP32 column sums for b2 and W3
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int c = c0 + 16 * hh;
        float h2[16];
        load_h2(c, h2);
        float v[16], w0[16], w1[16];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float d[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int jj = 8 * q + j;
                const float da2 = dy0 * F[L::W3 / 4 + c + jj] + dy1 * F[L::W3 / 4 + kHid + c + jj];
                d[j] = da2 * dsilu2(h2[jj]);
                v[jj] = d[j];
                const float a2 = silu2(h2[jj]);
                w0[jj] = dy0 * a2;
                w1[jj] = dy1 * a2;
            }
            *reinterpret_cast<uint4 *>(S + L::DH + tc_off(s, c + 8 * q, 2 * kHid)) =
                make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]), pack_bf16(d[6], d[7]));
        }
        const float r0 = warp_colsum16(v), r1 = warp_colsum16(w0), r2 = warp_colsum16(w1);
        if (lane < 16) {
            slot_add(0 * 32 + 16 * hh + lane, r0);
            slot_add(1 * 32 + 16 * hh + lane, r1);
            slot_add(2 * 32 + 16 * hh + lane, r2);
        }
    }
    // ---- da1 = dh2 W2 (M 128, N 64, K 64: W2 read MN-major) over H2's columns; dh1 =
    // da1 silu'(h1) into units 64..127 of DH; sums for b1 and W1u
    tc_publish();
    if (tid == 0) {
        tc_gemm(tm + L::cDA1, S, TcOp{L::DH, 2 * kHid, false}, TcOp{L::W2, kHid, true}, kHid, kHid);
        umma::commit(bar);
    }
    if (!tc_wait(bar, phase)) return false;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int c = c0 + 16 * hh;
        float h1[16], da1[16];
        load_h1(c, h1);
        tc_load16(tm + lane_base + L::cDA1 + c, da1);
        float g0[16], g1[16];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float d[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int jj = 8 * q + j;
                d[j] = da1[jj] * dsilu1(h1[jj]);
                da1[jj] = d[j];
                g0[jj] = d[j] * ux;
                g1[jj] = d[j] * uy;
            }
            *reinterpret_cast<uint4 *>(S + L::DH + tc_off(s, kHid + c + 8 * q, 2 * kHid)) =
                make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]), pack_bf16(d[6], d[7]));
        }
        const float r3 = warp_colsum16(da1), r4 = warp_colsum16(g0), r5 = warp_colsum16(g1);
        if (lane < 16) {
            slot_add(3 * 32 + 16 * hh + lane, r3);
            slot_add(4 * 32 + 16 * hh + lane, r4);
            slot_add(5 * 32 + 16 * hh + lane, r5);
        }
    }
    // ---- dz = dh1 W1z (N 32, K 64: W1z read MN-major) over dA1's columns; dW2 += dh2^T a1
    // and dW1z += dh1^T z from the stacked [dh2 | dh1], A1 and Z read MN-major (M 128
    // units, K 128 samples)
    tc_publish();
    if (tid == 0) {
        tc_gemm(tm + L::cDZ, S, TcOp{L::DH + kHid / 8 * 128, 2 * kHid, false}, TcOp{L::W1z, kLat, true}, kLat, kHid);
        tc_gemm(tm + L::cDW2, S, TcOp{L::DH, 2 * kHid, true}, TcOp{L::A1, kHid, true}, kHid, kSampC, !first);
        tc_gemm(tm + L::cDW1z, S, TcOp{L::DH, 2 * kHid, true}, TcOp{L::Z, kLat, true}, kLat, kSampC, !first);
        umma::commit(bar);
    }
    if (!last) load_latents(A, cbase + kSampC + s, wg, zv);  // the next chunk's, in flight during the MMAs
    if (!tc_wait(bar, phase)) return false;
    {
        float v[16];
        tc_load16(tm + lane_base + L::cDZ + 16 * wg, v);
        float *dst = expl ? A.dzout : A.dzs;
        if (valid && dst) {
            dst += (cbase + s) * kLat + 16 * wg;
            if (((uintptr_t)dst & 15u) == 0) {
                st_f4x4(dst, v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) dst[j] = v[j];
            }
        }
    }
    if (!last) return true;
    // gradient rows are 16-byte aligned (kGP = 6532 floats; dW2 at 2240, dW1z at 0)
    float *gp = A.gpart + (int64_t)blockIdx.x * kGP;
    if (s < kHid) {  // lanes 0..63: dW2[out = s][in]
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            float v[16];
            tc_load16(tm + lane_base + L::cDW2 + c0 + 16 * hh, v);
            st_f4x4(gp + oW2 + s * kHid + c0 + 16 * hh, v);
        }
    } else {  // lanes 64..127: dW1z[out = s - 64][in]
        float v[16];
        tc_load16(tm + lane_base + L::cDW1z + 16 * wg, v);
        st_f4x4(gp + oW1z + (s - kHid) * kLat + 16 * wg, v);
    }
    __syncthreads();
    // ---- the FP32 column sums: warps 4 wg .. 4 wg + 3 cover all samples of columns 32 wg ..
    for (int e = tid; e < 6 * kHid; e += 256) {
        const int q = e / kHid, c = e % kHid, w0 = 4 * (c / 32);
        float acc = 0.0f;
        for (int w = w0; w < w0 + 4; ++w) acc += F[L::Slots / 4 + (w * 6 + q) * 32 + (c % 32)];
        const int dst = q == 0 ? ob2 + c : q == 1 ? oW3 + c : q == 2 ? oW3 + kHid + c
                      : q == 3 ? ob1 + c : q == 4 ? oW1u + 2 * c : oW1u + 2 * c + 1;
        gp[dst] = acc;
    }
    if (tid < 3) {
        float acc = 0.0f;
        for (int w = 0; w < 4; ++w) acc += F[L::WS / 4 + w * 4 + tid];
        gp[tid < 2 ? ob3 + tid : kParams] = tid < 2 ? acc : acc * A.inv_batch;
    }
    return true;
}

// Training (backward = 1) or validation step over 256 samples per CTA in two
// chunks of 128 (two CTAs per SM: ~85 KB of shared memory, 256 tensor-memory
// columns each): the layer-1 latent block, layer 2 and the four backward products
// on the fifth-generation tensor cores (tcgen05.mma, BF16 operands in shared
// memory, FP32 accumulators in tensor memory, mbarrier completion with bounded
// waits); position block, biases, layer 3 and all column sums in FP32.  One CTA row
// of weight gradients per 256 samples: half the rows, and half the per-CTA set-up,
// of a CTA per chunk.
__global__ void __launch_bounds__(256, 2) k_ff_train(TrainArgs A)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar, idle;  // MMA completion; a barrier nothing arrives on (probe)
    __shared__ uint32_t tmem;
    using L = TrainTc;
    float *F = reinterpret_cast<float *>(tsm);
    int *I = reinterpret_cast<int *>(tsm);
    const int tid = threadIdx.x;

    // ---- samples, one per thread (both chunks): generated ones depend only on the
    // fit's fixed tables and run before the wait on the previous kernel (explicit ones
    // are read after it)
    const bool gen = A.zin == nullptr;
    if (gen) {
        const int64_t li = (int64_t)blockIdx.x * kSampCTA + tid;
        const bool valid = li < A.spec.count;
        int rc = 0;
        float ux = 0.f, uy = 0.f, tx = 0.f, ty = 0.f, scv = 1.0f, vp = 1.0f;
        if (valid) sample_of(A, li, rc, ux, uy, tx, ty, scv, vp);
        F[L::U / 4 + 2 * tid] = ux;
        F[L::U / 4 + 2 * tid + 1] = uy;
        F[L::T / 4 + 2 * tid] = tx;
        F[L::T / 4 + 2 * tid + 1] = ty;
        F[L::SV / 4 + tid] = scv * vp;
        I[L::RC / 4 + tid] = rc;
        I[L::OK / 4 + tid] = valid ? 1 : 0;
    }
    if (tid == 0) {
        umma::mbar_init(&bar, 1);
        umma::mbar_init(&idle, 1);
        umma::fence_mbar_init();
    }
    if (tid < 32) umma::tmem_alloc(&tmem, L::ncols);
    // ---- the previous kernel's results: weights, latents.  Only after the wait may the
    // next kernel (the step's update, which reads what the previous update wrote
    // before its own wait) begin launching.
    pdl_wait();
    pdl_launch_next();
    // ---- latents of this thread's sample of the first chunk (columns 16 wg .. 16 wg + 15),
    // in flight during the weight staging
    float zv[16];
    load_latents(A, (int64_t)blockIdx.x * kSampCTA + (tid & (kSampC - 1)), tid >> 7, zv);
    // ---- weights: the BF16 operands' shared-memory image (16-byte copies), FP32
    // small parameters
    for (int i = tid; i < kWImgBytes / 16; i += 256)
        reinterpret_cast<uint4 *>(tsm)[i] = reinterpret_cast<const uint4 *>(A.wimg)[i];
    if (tid < 2 * kHid) {
        F[L::W1u / 4 + tid] = A.params[oW1u + tid];
        F[L::W3 / 4 + tid] = A.params[oW3 + tid];
    }
    if (tid < kHid) {
        F[L::b1 / 4 + tid] = A.params[ob1 + tid];
        F[L::b2 / 4 + tid] = A.params[ob2 + tid];
    }
    if (tid < 2) F[L::b3 / 4 + tid] = A.params[ob3 + tid];
    if (!gen) {
        const int64_t li = (int64_t)blockIdx.x * kSampCTA + tid;
        const bool valid = li < A.spec.count;
        float ux = 0.f, uy = 0.f, tx = 0.f, ty = 0.f;
        if (valid) {
            ux = A.uin[2 * li];
            uy = A.uin[2 * li + 1];
            tx = A.tin ? A.tin[2 * li] : 0.f;
            ty = A.tin ? A.tin[2 * li + 1] : 0.f;
        }
        F[L::U / 4 + 2 * tid] = ux;
        F[L::U / 4 + 2 * tid + 1] = uy;
        F[L::T / 4 + 2 * tid] = tx;
        F[L::T / 4 + 2 * tid + 1] = ty;
        F[L::SV / 4 + tid] = 1.0f;
        I[L::RC / 4 + tid] = 0;
        I[L::OK / 4 + tid] = valid ? 1 : 0;
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tm = tmem;
    uint32_t phase = 0;
#pragma unroll 1
    for (int chunk = 0; chunk < kChunks; ++chunk) {
        // (a backward chunk loads the next one's latents itself)
        if (chunk > 0 && !A.backward)
            load_latents(A, (int64_t)blockIdx.x * kSampCTA + chunk * kSampC + (tid & (kSampC - 1)), tid >> 7, zv);
        if (!train_step(A, tsm, &bar, &idle, tm, phase, zv, chunk)) {
            // a completion wait gave up: flag it and drain (bounded) before freeing
            // the tensor memory
            if (tid == 0) {
                if (A.err) atomicExch(A.err, 1);
                umma::mbar_wait(&bar, phase, kWaitPolls);
            }
            break;
        }
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    if (tid < 32) umma::tmem_dealloc(tm, L::ncols);
}

// Launch with programmatic stream serialisation (PDL): the kernel may begin while
// the previous one of the stream finishes (see pdl_wait).
template <class... P, class... A>
static cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

cudaError_t ff_train_step(const TrainArgs &t, int64_t nsamples, cudaStream_t s, bool pdl)
{
    // two CTAs of ~85 KB per SM (tensor memory allows no more): the largest shared-memory carveout
    cudaError_t e = cudaFuncSetAttribute(k_ff_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TrainTc::bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ff_train, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (nsamples <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nsamples + kSampCTA - 1) / kSampCTA);
    if (pdl) return launch_pdl(k_ff_train, dim3(nb), dim3(256), TrainTc::bytes, s, t);
    k_ff_train<<<nb, 256, TrainTc::bytes, s>>>(t);
    return cudaGetLastError();
}

int64_t ff_gpart_stride() { return kGP; }
int64_t ff_train_blocks(int64_t nsamples) { return (nsamples + kSampCTA - 1) / kSampCTA; }

// grads[p] = sum over the CTA rows of gpart: a CTA takes 32 columns; its 8 row
// groups each sum a contiguous eighth of the rows in row order (loads in flight
// together), then the 8 partial sums are added in group order.  The order is
// fixed, so training stays bit-reproducible.
constexpr int kRedCols = 32, kRedGroups = 8;

__global__ void __launch_bounds__(kRedCols * kRedGroups) k_reduce_grads(const float *__restrict__ gpart, int64_t nblk,
                                                                       float *__restrict__ grads, float *__restrict__ loss)
{
    __shared__ float part[kRedGroups][kRedCols];
    const int c = threadIdx.x % kRedCols, g = threadIdx.x / kRedCols;
    const int p = blockIdx.x * kRedCols + c;  // parameter index; kParams is the loss
    const int64_t per = (nblk + kRedGroups - 1) / kRedGroups;
    const int64_t b0 = g * per, b1 = min(nblk, b0 + per);
    float acc = 0.0f;
    if (p <= kParams) {
#pragma unroll 16
        for (int64_t b = b0; b < b1; ++b) acc += gpart[b * kGP + p];
    }
    part[g][c] = acc;
    __syncthreads();
    if (g == 0 && p <= kParams) {
        float t = part[0][c];
#pragma unroll
        for (int q = 1; q < kRedGroups; ++q) t += part[q][c];
        if (p < kParams)
            grads[p] = t;
        else if (loss)
            *loss = t;
    }
}

cudaError_t ff_reduce_grads(const float *gpart, int64_t nblk, float *grads, float *loss, cudaStream_t s)
{
    k_reduce_grads<<<(kParams + 1 + kRedCols - 1) / kRedCols, kRedCols * kRedGroups, 0, s>>>(gpart, nblk, grads, loss);
    return cudaGetLastError();
}



// The rest of a training step in one launch: the weight gradients summed over the
// step's CTA rows (as k_reduce_grads: 32 columns per CTA, eight row groups in row
// order, then in group order), each latent's gradient over the step's samples of
// its cell in sample order (sample li of the step is sample offset + li of the
// sequence, whose cell is its index mod nrc), and the Adam update (Kingma & Ba
// 2015) of every parameter with its sum, refreshing the BF16 weight copies and the
// training kernel's operand image.  The summation orders are fixed, so training is
// bit-reproducible.
__global__ void __launch_bounds__(kRedCols * kRedGroups) k_step_update(StepUpdate U)
{
    constexpr int kWBlocks = (kParams + 1 + kRedCols - 1) / kRedCols;
    // the next training step may begin launching; this thread's parameter and Adam
    // moments (last written two kernels back) are read before the wait for the
    // step's gradients
    pdl_launch_next();
    int64_t mine = -1;
    if (blockIdx.x < kWBlocks) {
        const int p = blockIdx.x * kRedCols + threadIdx.x % kRedCols;
        if (threadIdx.x / kRedCols == 0 && p < kParams) mine = p;
    } else {
        const int64_t e = (int64_t)(blockIdx.x - kWBlocks) * blockDim.x + threadIdx.x;
        if (e < (int64_t)U.nrc * kLat) mine = kParams + e;
    }
    float m0 = 0.f, v0 = 0.f, p0 = 0.f;
    if (mine >= 0) {
        m0 = U.m[mine];
        v0 = U.v[mine];
        p0 = U.p[mine];
    }
    pdl_wait();
    auto adam_one = [&](int64_t i, float gi) {
        const float mi = U.b1 * m0 + (1.0f - U.b1) * gi;
        const float vi = U.b2 * v0 + (1.0f - U.b2) * gi * gi;
        U.m[i] = mi;
        U.v[i] = vi;
        const float lr = i < kParams ? U.lr_w : U.lr_z;
        const float pn = p0 - lr * (mi / U.bc1) / (sqrtf(vi / U.bc2) + U.eps);
        U.p[i] = pn;
        if (i >= oW1z && i < oW1z + kHid * kLat) {
            U.w1zb[i - oW1z] = to_bf16(pn);
            wimg_put(U.wimg, i, to_bf16(pn));
        }
        if (i >= oW2 && i < oW2 + kHid * kHid) {
            U.w2b[i - oW2] = to_bf16(pn);
            wimg_put(U.wimg, i, to_bf16(pn));
        }
    };
    if (blockIdx.x < kWBlocks) {
        __shared__ float part[kRedGroups][kRedCols];
        const int c = threadIdx.x % kRedCols, g = threadIdx.x / kRedCols;
        const int p = blockIdx.x * kRedCols + c;  // parameter index; kParams is the loss
        const int64_t per = (U.nblk + kRedGroups - 1) / kRedGroups;
        const int64_t b0 = g * per, b1 = min(U.nblk, b0 + per);
        float acc = 0.0f;
        if (p <= kParams) {
#pragma unroll 16
            for (int64_t b = b0; b < b1; ++b) acc += U.gpart[b * kGP + p];
        }
        part[g][c] = acc;
        __syncthreads();
        if (g == 0 && p <= kParams) {
            float t = part[0][c];
#pragma unroll
            for (int q = 1; q < kRedGroups; ++q) t += part[q][c];
            if (p < kParams)
                adam_one(p, t);
            else if (U.loss)
                *U.loss = t;
        }
        return;
    }
    const int64_t e = (int64_t)(blockIdx.x - kWBlocks) * blockDim.x + threadIdx.x;
    if (e >= (int64_t)U.nrc * kLat) return;
    const int c = (int)(e / kLat), k = (int)(e % kLat);
    int64_t li = ((int64_t)c - U.offset % U.nrc + U.nrc) % U.nrc;
    float acc = 0.0f;
    for (; li < U.count; li += U.nrc) acc += U.dzs[li * kLat + k];
    adam_one(kParams + e, acc);
}

cudaError_t ff_step_update(const StepUpdate &u, cudaStream_t s)
{
    constexpr int kWBlocks = (kParams + 1 + kRedCols - 1) / kRedCols;
    const int64_t nlat = (int64_t)u.nrc * kLat;
    const unsigned grid = (unsigned)(kWBlocks + (nlat + kRedCols * kRedGroups - 1) / (kRedCols * kRedGroups));
    return launch_pdl(k_step_update, dim3(grid), dim3(kRedCols * kRedGroups), 0, s, u);
}

// e_c = bf16(W1z) bf16(z_c) + b1 (FP32 accumulation): layer 1 without the position block
__global__ void k_embed(const float *p, const float *z, int nrc, float *ec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nrc * kHid) return;
    const int rc = (int)(i / kHid), col = (int)(i % kHid);
    float acc = 0.0f;
    for (int k = 0; k < kLat; ++k)
        acc = __fmaf_rn(__bfloat162float(to_bf16(p[oW1z + col * kLat + k])),
                        __bfloat162float(to_bf16(z[(int64_t)rc * kLat + k])), acc);
    ec[i] = acc + p[ob1 + col];
}

cudaError_t ff_embed(const float *params, const float *z, int nrc, float *ec, cudaStream_t s)
{
    const int64_t n = (int64_t)nrc * kHid;
    k_embed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, z, nrc, ec);
    return cudaGetLastError();
}

__global__ void k_flags(const unsigned *maxerr, int nrc, float tol, int *flags)
{
    const int rc = blockIdx.x * blockDim.x + threadIdx.x;
    if (rc < nrc) flags[rc] = __uint_as_float(maxerr[rc]) > tol ? 1 : 0;
}

cudaError_t ff_flags(const unsigned *maxerr, int nrc, float tol, int *flags, cudaStream_t s)
{
    k_flags<<<(nrc + 255) / 256, 256, 0, s>>>(maxerr, nrc, tol, flags);
    return cudaGetLastError();
}

// ================================================ learned shooting kernel
struct LearnSmem {
    __align__(128) unsigned char w2cm[kHid * kHid * 2];  // W2 / 2 [out][in], BF16, core-matrix layout (B operand)
    uint64_t mbar[2];     // per warpgroup: completion of its tensor-core MMAs
    uint64_t idle;        // an mbarrier nothing arrives on (the wait probe, a test aid)
    uint32_t tmem;        // tensor-memory base: 128 columns, 64 per warpgroup
    int wg_ok[8];         // per warp: the last wait completed
    int tc_dead[2];       // per warpgroup: a wait gave up; no more MMAs
    uint32_t pending[2];  // the phase a dead warpgroup still waits for
    // the tile's cell embedding per pair of hidden units (c, c + 1), halved (the block
    // forms v / 2, SiLU's argument); the shared constants come with the launch (NetConsts)
    float2 ec2[kHid / 2];  // {e_c, e_c+1} / 2
    float coef[kCoefStride];
    float4 coef2[kPeMax];  // b_q as {Re, Re, Im, Im}: both rays of a pair at once
    float sc;
    int rb[3], re[3];
    int nnear;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// SiLU of two hidden units at once, as silu_hw, from h = v / 2: h + h tanh(h) with
// the hardware tanh (one packed FMA).  The learned kernel forms h directly: every
// constant that enters a pre-activation (e_c, W1u, W2, b2) is staged halved, and
// halving is exact, so h equals 0.5 v of the unhalved evaluation bit for bit.
static_assert(kLayer2Hw, "the packed network block uses the hardware-tanh SiLU in both layers");
__device__ __forceinline__ float2 silu_half2(float2 h)
{
    return __ffma2_rn(h, make_float2(tanh_hw(h.x), tanh_hw(h.y)), h);
}

// One tile of a non-flagged cell: near stars exactly (FP32 recentred + Kahan,
// as the plain kernel), far field = float-pair b0 + series to order pe +
// network residual, then beta and the same binning epilogue.
// Near-field stars per compensated chunk (a tile's 3 x 3 block holds ~1.3 stars per
// ray at the learned workload's density; a chunk is padded with massless far stars):
// 4 with the network, 2 for the series alone (measured fastest for each).
template <bool NET>
constexpr int kNearChunk = NET ? 4 : 2;
constexpr int kTcChunk = 128;                            // rays per tensor-core MMA (M)
constexpr int kTcABytes = kTcChunk * kHid * 2;           // one warpgroup's A operand (16 KB)
constexpr int kTcSmem = 2 * kTcABytes;                   // the two A operands
constexpr size_t kLearnedDynSmem = kTcSmem > sizeof(ShootSmem<256>) ? kTcSmem : sizeof(ShootSmem<256>);

// LO: the ray offsets carry low parts (grids whose offsets are not exact floats,
// RayGrid lo); a separate instance so that the exact-offset tiles keep their
// registers.
template <bool NET, bool LO>
__device__ __forceinline__ void learned_tile(const LearnedArgs &L, int bx, int by, ShootSmem<256> &sm, TileShared &ts,
                                             LearnSmem &ls, unsigned char *abuf_all, uint32_t &phase)
{
    constexpr int NP = 4;
    constexpr int kTileY = 32;
    const ShootArgs &a = L.plain;
    const RayGrid &R = a.rays;
    const CellGrid &cg = L.cg;
    const int tid = threadIdx.x, tx = tid % kTileX, tg = tid / kTileX;
    const int i0 = bx * kTileX, j0 = by * kTileY;
    const int cx = bx / cg.ktx, cy = by / cg.kty, rc = cy * cg.ncx + cx;
    if (tid == 0) {
        double cxd = R.x0 + ((double)i0 + 0.5 * kTileX) * R.dx;
        double cyd = R.y0 + ((double)j0 + 0.5 * kTileY) * R.dy;
        float fcx = tile_centre(cxd, kTileX * R.dx, R.qx, R.qxinv);
        float fcy = tile_centre(cyd, kTileY * R.dy, R.qy, R.qyinv);
        double ex = (R.x0 + ((double)i0 + 0.5) * R.dx) - (double)fcx;
        double ey = (R.y0 + ((double)j0 + 0.5) * R.dy) - (double)fcy;
        double bxd = a.lens.a11 * (double)fcx + a.lens.a12 * (double)fcy;
        double byd = a.lens.a12 * (double)fcx + a.lens.a22 * (double)fcy;
        float bxh = (float)bxd, byh = (float)byd;
        ts.tc[0] = fcx;
        ts.tc[1] = fcy;
        ts.tc[2] = (float)ex;
        ts.tc[3] = (float)ey;
        ts.tc[4] = bxh;
        ts.tc[5] = byh;
        ts.tc[6] = (float)(bxd - (double)bxh);
        ts.tc[7] = (float)(byd - (double)byh);
        ts.tc[8] = (float)(ex - (double)ts.tc[2]);
        ts.tc[9] = (float)(ey - (double)ts.tc[3]);
        ts.sred[0] = ts.sred[1] = ts.sred[2] = 0u;
        const int ecx = cx + 1, ecy = cy + 1;
        int tot = 0;
        for (int d = -1; d <= 1; ++d) {
            const int row = (ecy + d) * cg.nx;
            ls.rb[d + 1] = L.cstart[row + ecx - 1];
            ls.re[d + 1] = L.cstart[row + ecx + 2];
            tot += ls.re[d + 1] - ls.rb[d + 1];
        }
        ls.nnear = tot;
        ls.sc = L.sc[rc];
    }
    if (tid < kCoefStride) ls.coef[tid] = L.coef[(int64_t)rc * kCoefStride + tid];
    if (tid < kPeMax) {
        const float re = L.coef[(int64_t)rc * kCoefStride + 4 + 2 * tid];
        const float im = L.coef[(int64_t)rc * kCoefStride + 5 + 2 * tid];
        ls.coef2[tid] = make_float4(re, re, im, im);
    }
    if (tid < kHid)  // e_c / 2 (exact)
        reinterpret_cast<float *>(&ls.ec2[tid >> 1])[tid & 1] = L.ec ? 0.5f * L.ec[(int64_t)rc * kHid + tid] : 0.0f;
    __syncthreads();

    // ray offsets from the tile centre: the high parts here, the low parts (LO) formed
    // inside the near-field loop
    float2 rx, ry[NP], px[NP], py[NP], Sx[NP], Sy[NP], Cx[NP], Cy[NP];
    const float cxf = ts.tc[0], cyf = ts.tc[1];
    if (LO) {
        float h, l, h1, l1;
        ray_offset((float)tx, ts.tc[2], ts.tc[8], R.dxh, R.dxl, h, l);
        rx = f2(h, h);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
            ray_offset(k0, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h, l);
            ray_offset(k1, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h1, l1);
            ry[p] = f2(h, h1);
            px[p] = py[p] = Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
        }
    } else {  // exact float offsets: e + k d with every step exact
        const float kx = (float)tx;
        const float dxr = __fmaf_rn(kx, R.dxh, ts.tc[2]);
        rx = f2(dxr, dxr);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
            ry[p] = f2(__fmaf_rn(k0, R.dyh, ts.tc[3]), __fmaf_rn(k1, R.dyh, ts.tc[3]));
            px[p] = py[p] = Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
        }
    }
    // ---- near field: the 3 x 3 block's stars (about 1.3 per tile at the learned
    // workload's density), staged 256 at a time and summed in compensated chunks
    // of kNearChunk<NET> stars, padded with massless far stars
    const int nnear = ls.nnear;
    for (int base = 0; base < nnear; base += 256) {
        constexpr int C = kNearChunk<NET>;
        const int cnt = min(256, nnear - base), cntp = (cnt + C - 1) / C * C;
        __syncthreads();
        if (tid < cntp) {
            float4 q = make_float4(kPadCoord, kPadCoord, 0.0f, 0.0f);
            if (tid < cnt) {
                int k = base + tid;
                const int n0 = ls.re[0] - ls.rb[0], n1 = ls.re[1] - ls.rb[1];
                const int idx = k < n0 ? ls.rb[0] + k : (k < n0 + n1 ? ls.rb[1] + (k - n0) : ls.rb[2] + (k - n0 - n1));
                q = L.cstars[idx];
            }
            const float nx = __fsub_rn(cxf, q.x), ny = __fsub_rn(cyf, q.y);
            sm.st.q[0][tid] = make_float4(nx, nx, ny, ny);
            sm.st.mm[0][tid] = f2(q.z, q.z);
        }
        __syncthreads();
        const float4 *Q = sm.st.q[0];
        const float2 *M = sm.st.mm[0];
        {
            float2 rxl = f2(0.f, 0.f), ryl[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) ryl[p] = f2(0.f, 0.f);
            if (LO) {
                float h, l, h1, l1;
                ray_offset((float)tx, ts.tc[2], ts.tc[8], R.dxh, R.dxl, h, l);
                rxl = f2(l, l);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
                    ray_offset(k0, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h, l);
                    ray_offset(k1, ts.tc[3], ts.tc[9], R.dyh, R.dyl, h1, l1);
                    ryl[p] = f2(l, l1);
                }
            }
            for (int k0 = 0; k0 < cntp; k0 += C) {
#pragma unroll
                for (int k = k0; k < k0 + C; ++k) {
                    const float4 q = Q[k];
                    const float2 m2 = M[k];
                    const float2 dx = LO ? __fadd2_rn(__fadd2_rn(rx, f2(q.x, q.y)), rxl) : __fadd2_rn(rx, f2(q.x, q.y));
                    const float2 dx2 = __fmul2_rn(dx, dx);
                    const float2 nyv = f2(q.z, q.w);
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const float2 dy = LO ? __fadd2_rn(__fadd2_rn(ry[p], nyv), ryl[p]) : __fadd2_rn(ry[p], nyv);
                        const float2 r2 = __ffma2_rn(dy, dy, dx2);
                        const float2 inv = f2(rcp_approx(r2.x), rcp_approx(r2.y));
                        const float2 f = __fmul2_rn(m2, inv);
                        px[p] = __ffma2_rn(f, dx, px[p]);
                        py[p] = __ffma2_rn(f, dy, py[p]);
                    }
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    kahan2(Sx[p], Cx[p], px[p]);
                    kahan2(Sy[p], Cy[p], py[p]);
                    px[p] = py[p] = f2(0.f, 0.f);
                }
            }
        }
    }
    __syncthreads();  // star stages dead; the region now holds the network outputs

    // ---- network residual for the tile's 2048 rays (warp w: rays 256w .. 256w+255)
    // the network's outputs (+ b3) for this thread's own rays, ray k at yv[2 k], yv[2 k + 1]
    float yv[4 * NP];
    const int ioff = (bx % cg.ktx) * kTileX, joff = (by % cg.kty) * kTileY;
    const float inv_cx = 1.0f / (float)(kTileX * cg.ktx), inv_cy = 1.0f / (float)(kTileY * cg.kty);
    if (NET) {
        // Two warpgroups; warpgroup wg takes the 128-ray chunks wg, wg + 2, ...  Each
        // thread writes its ray's layer-1 activations (BF16) as row t of the
        // warpgroup's A operand; one thread issues h2 = A W2^T on the tensor cores
        // (tcgen05.mma, M = 128, N = 64, K = 64 in four K = 16 steps, FP32
        // accumulator in tensor memory) and commits to the warpgroup's mbarrier;
        // then each thread reads its ray's 64 accumulators back and finishes SiLU
        // and layer 3 in registers.
        const int warp = tid >> 5, lane = tid & 31, wg = warp >> 2, t = tid & 127;
        unsigned char *abuf = abuf_all + wg * kTcABytes;
        const uint32_t dcol = ls.tmem + (uint32_t)(wg * kHid);
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        constexpr uint32_t idesc = umma::idesc_bf16(kTcChunk, kHid);
#pragma unroll 1
        for (int k = 0; k < 2 * NP; ++k) {  // chunk k: ray k of each thread of the warpgroup
            const int row = tg * 2 * NP + k;  // the ray's row in the tile (its column is tx)
            float y0 = 0.0f, y1 = 0.0f;
            if (!ls.tc_dead[wg]) {
                const float ux = (float)(2 * (ioff + tx) + 1) * inv_cx - 1.0f;
                const float uy = (float)(2 * (joff + row) + 1) * inv_cy - 1.0f;
                const float2 uxx = make_float2(ux, ux), uyy = make_float2(uy, uy);
#pragma unroll
                for (int k8 = 0; k8 < kHid / 8; ++k8) {
                    uint32_t pk[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {  // units 8 k8 + 2 q and + 1
                        const float2 e = ls.ec2[4 * k8 + q];
                        const float4 w = L.net.w1u[4 * k8 + q];
                        // (e_c + W1u[.][0] ux + W1u[.][1] uy) / 2, then SiLU, for both units
                        float2 v = __ffma2_rn(make_float2(w.x, w.y), uxx, e);
                        v = __ffma2_rn(make_float2(w.z, w.w), uyy, v);
                        const float2 a = silu_half2(v);
                        pk[q] = pack_bf16(a.x, a.y);
                    }
                    *reinterpret_cast<uint4 *>(abuf + umma::cm_offset(t, k8 * 8)) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
                umma::fence_async_smem();
                umma::fence_before();
                umma::wg_sync(wg);
                umma::fence_after();
                if (t == 0) {
#pragma unroll
                    for (int ks = 0; ks < kHid / 16; ++ks)
                        umma::mma_bf16(dcol, umma::desc(umma::smem_addr(abuf) + ks * 256, 128, 1024),
                                       umma::desc(umma::smem_addr(ls.w2cm) + ks * 256, 128, 1024), idesc,
                                       ks > 0 ? 1u : 0u);
                    umma::commit(&ls.mbar[wg]);
                }
                // (the wait probe, a test aid, polls ls.idle instead: the wait runs out and
                // the warpgroup takes the failure path below)
                const bool ok = __all_sync(0xffffffffu, L.wait_probe ? umma::mbar_wait(&ls.idle, 0, kProbePolls)
                                                                     : umma::mbar_wait(&ls.mbar[wg], phase, kWaitPolls));
                if (lane == 0) ls.wg_ok[warp] = ok ? 1 : 0;
                umma::wg_sync(wg);
                const bool wg_ok = ls.wg_ok[4 * wg] && ls.wg_ok[4 * wg + 1] && ls.wg_ok[4 * wg + 2] &&
                                   ls.wg_ok[4 * wg + 3];
                if (wg_ok) {
                    phase ^= 1u;
                    umma::fence_after();
                    // layer 2's bias and SiLU, and layer 3, two units at a time (even and
                    // odd units summed apart, then added)
                    float2 y0p = make_float2(0.0f, 0.0f), y1p = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int c0 = 0; c0 < kHid; c0 += 16) {
                        uint32_t acc[16];
                        umma::ld16(dcol + lane_base + (uint32_t)c0, acc);
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            const float4 qa = L.net.l2p[(c0 + j) >> 1];
                            const float2 qb = L.net.l2q[(c0 + j) >> 1];
                            const float2 a2 = silu_half2(__fadd2_rn(
                                make_float2(__uint_as_float(acc[j]), __uint_as_float(acc[j + 1])), make_float2(qa.x, qa.y)));
                            y0p = __ffma2_rn(make_float2(qa.z, qa.w), a2, y0p);
                            y1p = __ffma2_rn(qb, a2, y1p);
                        }
                    }
                    y0 = y0p.x + y0p.y;
                    y1 = y1p.x + y1p.y;
                } else if (t == 0) {
                    // the MMAs never reported completion: stop using the tensor path,
                    // remember the phase to drain before tensor memory is freed
                    ls.tc_dead[wg] = 1;
                    ls.pending[wg] = phase;
                    atomicExch(L.err, 1);
                }
                umma::fence_before();
                umma::wg_sync(wg);  // accumulators read and A consumed before the next chunk
            }
            yv[2 * k] = y0 + L.net.b3[0];
            yv[2 * k + 1] = y1 + L.net.b3[1];
        }
    }

    // ---- far field and beta per ray, the two rays of each pair (rows 2p and 2p + 1 of
    // column tx) in the two lanes of f32x2 registers: the same operations per ray as a
    // scalar loop, x - y as fma(y, -1, x) (one rounding, as a subtraction)
    float bxh[2 * NP], byh[2 * NP], bxl[2 * NP], byl[2 * NP];
    {
        const float2 m1 = make_float2(-1.0f, -1.0f);
        auto sub2 = [&](float2 x, float2 y) { return __ffma2_rn(y, m1, x); };
        auto two_sum2 = [&](float2 a, float2 b, float2 &s, float2 &e) {  // Knuth's TwoSum per lane
            const float2 x = __fadd2_rn(a, b), bb = sub2(x, a);
            e = __fadd2_rn(sub2(a, sub2(x, bb)), sub2(b, bb));
            s = x;
        };
        auto dup = [](float x) { return make_float2(x, x); };
        const float uxr = (float)(2 * (ioff + tx) + 1) * inv_cx - 1.0f;
        const float2 vx = dup(uxr * 0.70710678f);
        const float2 tc4 = dup(ts.tc[4]), tc5 = dup(ts.tc[5]), tc6 = dup(ts.tc[6]), tc7 = dup(ts.tc[7]);
        const float2 nb0x = dup(-ls.coef[0]), b0y = dup(ls.coef[1]), b1x = dup(ls.coef[2]), b1y = dup(ls.coef[3]);
        const float2 fa11 = dup(a.lens.fa11), fa12 = dup(a.lens.fa12), fa22 = dup(a.lens.fa22);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int jl = tg * 2 * NP + 2 * p;  // the pair's first row in the tile
            const float uy0 = (float)(2 * (joff + jl) + 1) * inv_cy - 1.0f;
            const float uy1 = (float)(2 * (joff + jl + 1) + 1) * inv_cy - 1.0f;
            const float2 vy = make_float2(uy0 * 0.70710678f, uy1 * 0.70710678f);
            const float2 nvy = make_float2(-vy.x, -vy.y);
            // T = sum_{q=1}^{pe} b_q v^q + v^(pe+1) q_net, q_net = s_c (network output) or 0:
            // Horner with q_net as the innermost coefficient; (ar, ai) = T's real and
            // imaginary parts for the two rays
            float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
            if (L.use_net) {
                ar = make_float2(ls.sc * yv[4 * p], ls.sc * yv[4 * p + 2]);
                ai = make_float2(ls.sc * yv[4 * p + 1], ls.sc * yv[4 * p + 3]);
            }
            auto cmul2 = [&]() {  // (ar + i ai) (vx + i vy)
                const float2 t = __fmul2_rn(ar, vx), u = __fmul2_rn(ar, vy);
                ar = __ffma2_rn(ai, nvy, t);
                ai = __ffma2_rn(ai, vx, u);
            };
            cmul2();
            for (int q = L.pe; q >= 1; --q) {
                const float4 c = ls.coef2[q - 1];
                ar = __fadd2_rn(ar, make_float2(c.x, c.y));
                ai = __fadd2_rn(ai, make_float2(c.z, c.w));
                cmul2();
            }
            // A delta from the offsets' high parts: the low parts (2^-24 of an offset)
            // matter only inside the near-field sum, next to a star
            const float2 lx = __ffma2_rn(fa11, rx, __fmul2_rn(fa12, ry[p]));
            const float2 ly = __ffma2_rn(fa12, rx, __fmul2_rn(fa22, ry[p]));
            // alpha_far = (Re F, -Im F) + residual;  F = b0 + T
            float2 th, tl, t2, small, h, l;
            two_sum2(tc4, __fmul2_rn(Sx[p], m1), th, tl);
            two_sum2(th, nb0x, th, t2);
            small = __fadd2_rn(__fadd2_rn(tc6, Cx[p]), lx);
            small = sub2(small, __fadd2_rn(b1x, ar));
            tl = __fadd2_rn(__fadd2_rn(tl, t2), small);
            two_sum2(th, tl, h, l);
            bxh[2 * p] = h.x, bxh[2 * p + 1] = h.y, bxl[2 * p] = l.x, bxl[2 * p + 1] = l.y;
            two_sum2(tc5, __fmul2_rn(Sy[p], m1), th, tl);
            two_sum2(th, b0y, th, t2);
            small = __fadd2_rn(__fadd2_rn(tc7, Cy[p]), ly);
            small = __fadd2_rn(small, __fadd2_rn(b1y, ai));
            tl = __fadd2_rn(__fadd2_rn(tl, t2), small);
            two_sum2(th, tl, h, l);
            byh[2 * p] = h.x, byh[2 * p + 1] = h.y, byl[2 * p] = l.x, byl[2 * p + 1] = l.y;
        }
    }

    // ---- binning (the epilogue of the plain kernel)
    const int ix = i0 + tx;
    const bool col_ok = ix < R.nx;
    __syncthreads();
    hist_zero(sm.hist);
    if (tid == 0) {
        ts.win[0] = pair_axis_rough(bxh[0], a.bin.ax) - kWin / 2;
        ts.win[1] = pair_axis_rough(byh[0], a.bin.ay) - kWin / 2;
    }
    __syncthreads();
    WinHist W{sm.hist, ts.win[0], ts.win[1]};
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
    stats_add_block(nb, no, nn, ts.sred, a.stats);
}

// NET: the network on the tensor cores (tcgen05; 128 tensor-memory columns and the
// two A operands in dynamic shared memory, in the same bytes as the star stage and
// window); without it (the series alone) the kernel carries no tensor-core code.
template <int NRP, bool NET, bool LO>
// Four CTAs per SM (64 registers, ~280 bytes of spills per thread; tensor memory
// holds four CTAs' 128 columns): eight warps per scheduler hide the latency of the
// 128 hardware tanh per ray.  Measured per 32768^2-ray map: two CTAs per SM 0.060 s,
// three 0.056 s (when first measured); three 44.8 ms, four 44.0 ms with the current
// network block, and 13.2 -> 11.8 ms for the order-16 series alone.
__global__ void __launch_bounds__(kThreads, 4) k_shoot_learned(LearnedArgs L)
{
    __shared__ TileShared ts;
    __shared__ __align__(128) LearnSmem ls;
    __shared__ long long s_item;
    // dynamic: the star stage and window of the tile phases without tensor-core work,
    // and (NET) the two A operands of the network phase in the same bytes
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    ShootSmem<256> &sm = *reinterpret_cast<ShootSmem<256> *>(dyn_smem);
    unsigned char *tc_abuf = dyn_smem;
    const int tid = threadIdx.x;
    uint32_t phase = 0;  // completed MMA batches of this thread's warpgroup, mod 2
    if (NET) {
        for (int i = tid; i < kHid * kHid; i += kThreads)
            *reinterpret_cast<__nv_bfloat16 *>(ls.w2cm + umma::cm_offset(i / kHid, i % kHid)) =
                __float2bfloat16_rn(0.5f * __bfloat162float(L.w2b[i]));  // W2 / 2 (exact)
        if (tid < 2) ls.tc_dead[tid] = 0;
        if (tid == 0) {
            umma::mbar_init(&ls.mbar[0], 1);
            umma::mbar_init(&ls.mbar[1], 1);
            umma::mbar_init(&ls.idle, 1);
            umma::fence_mbar_init();
        }
        if (tid < 32) umma::tmem_alloc(&ls.tmem, 2 * kHid);
        umma::fence_async_smem();  // W2 is read by the tensor cores
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
    }
    const int ntx = (L.plain.rays.nx + kTileX - 1) / kTileX;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (long long)atomicAdd(L.counter, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= L.nitems) break;
        const int tile = L.items[item];
        const int bx = tile % ntx, by = tile / ntx;
        const int rc = (by / L.cg.kty) * L.cg.ncx + bx / L.cg.ktx;
        if (L.flags[rc])
            shoot_tile<4, 256, false, NRP, 1, LO ? 2 : 1>(L.plain, bx, by, sm, ts);
        else
            learned_tile<NET, LO>(L, bx, by, sm, ts, ls, tc_abuf, phase);
    }
    if (NET) {
        // a warpgroup that gave up on a wait drains its MMAs (again bounded) before
        // the tensor memory is freed
        if ((tid & 127) == 0 && ls.tc_dead[tid >> 7]) umma::mbar_wait(&ls.mbar[tid >> 7], ls.pending[tid >> 7], kWaitPolls);
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid < 32) umma::tmem_dealloc(ls.tmem, 2 * kHid);
    }
}

// Dynamic shared memory for the tensor-core operands, and the largest shared-memory
// carveout for three CTAs of ~60 KB per SM.
template <class K>
static cudaError_t learned_attributes(K kernel)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLearnedDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

static_assert(kNetPairs * 2 == kHid, "NetConsts holds one entry per pair of hidden units");
static_assert(sizeof(LearnedArgs) <= 4096, "the learned kernel's parameters (NetConsts included) stay within 4 KB");

void ff_net_consts(const float *p, NetConsts *c)
{
    for (int P = 0; P < kNetPairs; ++P) {
        const int u = 2 * P;
        c->w1u[P] = make_float4(0.5f * p[oW1u + 2 * u], 0.5f * p[oW1u + 2 * (u + 1)], 0.5f * p[oW1u + 2 * u + 1],
                                0.5f * p[oW1u + 2 * (u + 1) + 1]);
        c->l2p[P] = make_float4(0.5f * p[ob2 + u], 0.5f * p[ob2 + u + 1], p[oW3 + u], p[oW3 + u + 1]);
        c->l2q[P] = make_float2(p[oW3 + kHid + u], p[oW3 + kHid + u + 1]);
    }
    c->b3[0] = p[ob3];
    c->b3[1] = p[ob3 + 1];
}

cudaError_t ff_learned_grid(int *grid)
{
    // The persistent grid takes the resident CTAs per SM of the kernel without
    // tensor-core code (four: launch-bounded to 64 registers per thread).  The
    // tensor-core variant has the same register limit and fits four CTAs in shared
    // and tensor memory, though the occupancy query has reported fewer for it; CTAs
    // beyond those resident only find the shared work queue empty.
    int per_sm = 0, per_sm1 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shoot_learned<0, false, false>, kThreads,
                                                                  sizeof(ShootSmem<256>));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, k_shoot_learned<1, false, false>, kThreads,
                                                      sizeof(ShootSmem<256>));
    if (e != cudaSuccess) return e;
    per_sm = per_sm < per_sm1 ? per_sm : per_sm1;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *grid = nsm * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

template <int NRP, bool LO>
static cudaError_t launch_learned_t(const LearnedArgs &L, unsigned g, cudaStream_t s)
{
    if (L.use_net) {
        cudaError_t e = learned_attributes(k_shoot_learned<NRP, true, LO>);
        if (e != cudaSuccess) return e;
        k_shoot_learned<NRP, true, LO><<<g, kThreads, kLearnedDynSmem, s>>>(L);
    } else {
        k_shoot_learned<NRP, false, LO><<<g, kThreads, sizeof(ShootSmem<256>), s>>>(L);
    }
    return cudaGetLastError();
}

template <int NRP>
static cudaError_t launch_learned(const LearnedArgs &L, unsigned g, cudaStream_t s)
{
    return L.plain.rays.lo ? launch_learned_t<NRP, true>(L, g, s) : launch_learned_t<NRP, false>(L, g, s);
}

cudaError_t ff_shoot_learned(const LearnedArgs &L, int grid, int fma_pairs, cudaStream_t s)
{
    const int64_t g = L.nitems < grid ? (L.nitems > 0 ? L.nitems : 1) : grid;
    return fma_pairs ? launch_learned<1>(L, (unsigned)g, s) : launch_learned<0>(L, (unsigned)g, s);
}

}  // namespace mlens
