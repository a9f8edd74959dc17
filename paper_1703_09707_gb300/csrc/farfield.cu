// farfield.cu -- kernels of the learned-far-field variant (see farfield.h):
// cell CSR of the stars, FP64 local-expansion coefficients of the far field,
// network training / validation on BF16 tensor cores, and the persistent
// shooting kernel that evaluates near field + series + network per ray and
// falls back to the exact direct sum on flagged cells.
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

// ===================================================== FP64 coefficients
// One warp per ray cell, eight cells per CTA sharing each staged chunk of stars.
// b_0 (the far field's value at the centre, ~30 theta_E, needed to ~1e-9) is
// formed entirely in FP64.  For p >= 1 the terms -(m/s) w^(p+1) are formed in
// FP32 from the FP64 w (relative error ~p 6e-8 per term, far below what the
// series needs) and accumulated in FP64, so the sums keep FP64 accuracy while
// the per-term work moves to the FP32 pipe.
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
__device__ __forceinline__ DF df_rcp(DF a)
{
    const float y = __frcp_rn(a.h);           // relative error <= 2^-24
    const DF ay = df_mulf(a, y);              // ~1
    const DF r = df_add({1.0f, 0.0f}, {-ay.h, -ay.l});  // 1 - a y, ~2^-24
    return df_norm(y, __fmul_rn(y, r.h));     // y (1 + r): error ~2^-47
}

__global__ void __launch_bounds__(256) k_coeffs(const float4 *stars, const int *scell, int64_t n, CellGrid g, int pt,
                                                double scale, double *out)
{
    // One warp per ray cell.  Per far star: the order-0 term -m / (z_k - z_c) in
    // double-float arithmetic on the FP32 pipe, summed per lane over each stage's
    // stars and added to an FP64 accumulator once per stage; w = s / (z_k - z_c)
    // in FP32 and the higher orders t_p = t_0 w^p by an FP32 recurrence into
    // per-lane FP32 partials, summed across the warp after each 256-star stage,
    // lane p adding coefficient p's stage sum to its FP64 accumulator.
    __shared__ float4 sq[256];
    __shared__ int scl[256];
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
    double b0r = 0.0, b0i = 0.0;    // order 0, this lane's stars
    double accr = 0.0, acci = 0.0;  // lane p (1 <= p <= pt): coefficient p, all stages
    for (int64_t s0 = 0; s0 < n; s0 += 256) {
        const int cnt = (int)min((int64_t)256, n - s0);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            sq[threadIdx.x] = stars[s0 + threadIdx.x];
            scl[threadIdx.x] = scell[s0 + threadIdx.x];
        }
        __syncthreads();
        if (!ok) continue;
        float pr[kPtMax], pi[kPtMax];
#pragma unroll
        for (int p = 0; p < kPtMax; ++p) pr[p] = pi[p] = 0.0f;
        DF sr = {0.0f, 0.0f}, si = {0.0f, 0.0f};
        for (int k = lane; k < cnt; k += 32) {
            const int c = scl[k];
            if (c >= 0) {
                const int sx = c % g.nx, sy = c / g.nx;
                if (sx - ex <= 1 && ex - sx <= 1 && sy - ey <= 1 && ey - sy <= 1) continue;  // near star
            }
            const float4 q = sq[k];
            const DF dx = df_add(df_two_sum(q.x, -zxh), {-zxl, 0.0f});
            const DF dy = df_add(df_two_sum(q.y, -zyh), {-zyl, 0.0f});
            const DF inv = df_rcp(df_add(df_mul(dx, dx), df_mul(dy, dy)));
            const DF mi = df_mulf(inv, q.z);
            const DF tr = df_mul(mi, dx), ti = df_mul(mi, dy);  // -m/(z_k - z_c) = (-tr, ti)
            sr = df_add(sr, {-tr.h, -tr.l});
            si = df_add(si, ti);
            const float si_s = __fmul_rn(inv.h, fscale);
            const float fwr = __fmul_rn(dx.h, si_s), fwi = -__fmul_rn(dy.h, si_s);  // s / (z_k - z_c)
            float fr = -tr.h, fi = ti.h;
#pragma unroll
            for (int p = 0; p < kPtMax; ++p) {
                const float nr = fr * fwr - fi * fwi, ni = fr * fwi + fi * fwr;
                fr = nr;
                fi = ni;
                pr[p] += fr;
                pi[p] += fi;
            }
        }
        b0r += (double)sr.h + (double)sr.l;
        b0i += (double)si.h + (double)si.l;
#pragma unroll
        for (int p = 0; p < kPtMax; ++p) {
            float r = pr[p], i = pi[p];
            for (int o = 16; o; o >>= 1) {
                r += __shfl_xor_sync(0xffffffffu, r, o);
                i += __shfl_xor_sync(0xffffffffu, i, o);
            }
            if (lane == p + 1) {
                accr += (double)r;
                acci += (double)i;
            }
        }
    }
    if (!ok) return;
    for (int o = 16; o; o >>= 1) {
        b0r += __shfl_xor_sync(0xffffffffu, b0r, o);
        b0i += __shfl_xor_sync(0xffffffffu, b0i, o);
    }
    double *dst = out + (int64_t)rc * (pt + 1) * 2;
    if (lane == 0) {
        dst[0] = b0r;
        dst[1] = b0i;
    } else if (lane <= pt) {
        dst[2 * lane] = accr;
        dst[2 * lane + 1] = acci;
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

__global__ void k_prep_bf16(const float *p, __nv_bfloat16 *w1zb, __nv_bfloat16 *w2b, __nv_bfloat16 *w2tb,
                            __nv_bfloat16 *w1ztb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kHid) {
        const int o = i / kHid, k = i % kHid;
        const __nv_bfloat16 v = to_bf16(p[oW2 + i]);
        w2b[i] = v;
        w2tb[k * kHid + o] = v;
    }
    if (i < kHid * kLat) {
        const int o = i / kLat, k = i % kLat;
        const __nv_bfloat16 v = to_bf16(p[oW1z + i]);
        w1zb[i] = v;
        w1ztb[k * kHid + o] = v;
    }
}

cudaError_t ff_prep_bf16(const float *params, __nv_bfloat16 *w1zb, __nv_bfloat16 *w2b, __nv_bfloat16 *w2tb,
                         __nv_bfloat16 *w1ztb, cudaStream_t s)
{
    k_prep_bf16<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(params, w1zb, w2b, w2tb, w1ztb);
    return cudaGetLastError();
}

// ===================================================== training kernel
// Shared-memory plan (BF16 unless noted), leading dimensions padded by 8.
constexpr int kLdZ = kLat + 8;   // 40
constexpr int kLdH = kHid + 8;   // 72
constexpr int kSampW = 16;       // samples per warp
constexpr int kSampC = 128;      // samples per CTA
constexpr int kLdT = kSampC + 8; // 136

constexpr int kGP = kParams + 2;  // gpart row: the parameters' gradients, then the loss

struct TrainSmemLayout {
    static constexpr int W1z = 0;                          // [64][40]
    static constexpr int W2 = W1z + kHid * kLdZ;           // [64][72] (n=out, k=in)
    static constexpr int W2T = W2 + kHid * kLdH;           // [64][72] (n=in, k=out)
    static constexpr int W1zT = W2T + kHid * kLdH;         // [32][72] (n=in, k=out)
    static constexpr int Warp = W1zT + kLat * kLdH;        // per warp: Z[16][40], A1, DH2, DH1 [16][72]
    static constexpr int WarpSize = kSampW * kLdZ + 3 * kSampW * kLdH;
    static constexpr int A1T = Warp + 8 * WarpSize;        // [64][136] (in, sample)
    static constexpr int DH2T = A1T + kHid * kLdT;         // [64][136] (out, sample)
    static constexpr int ZT = DH2T + kHid * kLdT;          // [32][136]
    static constexpr int DH1T = ZT + kLat * kLdT;          // [64][136]
    static constexpr int EndBf = DH1T + kHid * kLdT;
    // FP32 block after the BF16 block
    static constexpr int fW1u = 0, fb1 = 128, fb2 = 192, fW3 = 256, fb3 = 384, fdb1 = 388, fdb2 = 452;
    static constexpr int fWarp = 516;  // per warp: u[16][2], t[16][2], sc[16]
    static constexpr int fWarpSize = 80;
    // per warp gradient slots, summed over the warps in a fixed order:
    // W3 [128] at 0, b3 [2] at 128, W1u [128] at 130, b1 [64] at 258, b2 [64] at 322, loss at 386
    static constexpr int fWG = fWarp + 8 * fWarpSize;
    static constexpr int kWG = 388;
    static constexpr int EndF = fWG + 8 * kWG;
    static constexpr size_t bytes = (size_t)EndBf * 2 + (size_t)EndF * 4 + 8 * 16 * 4 * 2;
};

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
    // q(v) at v = u / sqrt(2) by Horner
    const float vr = ux * 0.70710678f, vi = uy * 0.70710678f;
    const float *b = A.tail + (int64_t)rc * 2 * (A.pt - A.pe);
    float ar = b[2 * (A.pt - A.pe - 1)], ai = b[2 * (A.pt - A.pe - 1) + 1];
    for (int p = A.pt - 1; p > A.pe; --p) {
        const float nr = ar * vr - ai * vi + b[2 * (p - A.pe - 1)];
        const float ni = ar * vi + ai * vr + b[2 * (p - A.pe - 1) + 1];
        ar = nr;
        ai = ni;
    }
    scv = A.sc[rc];
    tx = ar / scv;
    ty = ai / scv;
    vp = powf(vr * vr + vi * vi, 0.5f * (float)(A.pe + 1));
}

__global__ void __launch_bounds__(256, 1) k_ff_train(TrainArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using L = TrainSmemLayout;
    __nv_bfloat16 *sb = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    float *sf = reinterpret_cast<float *>(smem_raw + (size_t)L::EndBf * 2);
    int *si = reinterpret_cast<int *>(sf + L::EndF);  // per warp: rc[16], valid[16]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;

    // ---- weights into shared memory
    for (int i = tid; i < kHid * kLat; i += 256) sb[L::W1z + (i / kLat) * kLdZ + i % kLat] = A.w1zb[i];
    for (int i = tid; i < kHid * kHid; i += 256) {
        sb[L::W2 + (i / kHid) * kLdH + i % kHid] = A.w2b[i];
        sb[L::W2T + (i / kHid) * kLdH + i % kHid] = A.w2tb[i];
    }
    for (int i = tid; i < kLat * kHid; i += 256) sb[L::W1zT + (i / kHid) * kLdH + i % kHid] = A.w1ztb[i];
    for (int i = tid; i < 128; i += 256) {
        sf[L::fW1u + i] = A.params[oW1u + i];
        sf[L::fW3 + i] = A.params[oW3 + i];
    }
    if (tid < 64) {
        sf[L::fb1 + tid] = A.params[ob1 + tid];
        sf[L::fb2 + tid] = A.params[ob2 + tid];
    }
    if (tid < 2) sf[L::fb3 + tid] = A.params[ob3 + tid];

    // ---- samples of this warp
    float *wu = sf + L::fWarp + warp * L::fWarpSize;  // u[16][2] at 0, t[16][2] at 32, s_c |v|^(pe+1) [16] at 64
    int *wrc = si + warp * 32;                        // rc[16], valid[16]
    const int64_t cbase = (int64_t)blockIdx.x * kSampC + warp * kSampW;
    const bool expl = A.zin != nullptr;
    if (lane < kSampW) {
        const int64_t li = cbase + lane;
        const bool valid = li < A.spec.count;
        int rc = 0;
        float ux = 0.f, uy = 0.f, tx = 0.f, ty = 0.f, scv = 1.0f, vp = 1.0f;
        if (valid) {
            if (expl) {
                ux = A.uin[2 * li];
                uy = A.uin[2 * li + 1];
                tx = A.tin ? A.tin[2 * li] : 0.f;
                ty = A.tin ? A.tin[2 * li + 1] : 0.f;
            } else {
                sample_of(A, li, rc, ux, uy, tx, ty, scv, vp);
            }
        }
        wu[2 * lane] = ux;
        wu[2 * lane + 1] = uy;
        wu[32 + 2 * lane] = tx;
        wu[32 + 2 * lane + 1] = ty;
        wu[64 + lane] = scv * vp;
        wrc[lane] = rc;
        wrc[16 + lane] = valid ? 1 : 0;
    }
    __syncthreads();

    __nv_bfloat16 *sZ = sb + L::Warp + warp * L::WarpSize;
    __nv_bfloat16 *sA1 = sZ + kSampW * kLdZ;
    __nv_bfloat16 *sDH2 = sA1 + kSampW * kLdH;
    __nv_bfloat16 *sDH1 = sDH2 + kSampW * kLdH;
    for (int e = lane; e < kSampW * kLat; e += 32) {
        const int r = e >> 5, k = e & 31;
        float v = 0.0f;
        if (wrc[16 + r]) v = expl ? A.zin[(cbase + r) * kLat + k] : A.z[(int64_t)wrc[r] * kLat + k];
        const __nv_bfloat16 b = to_bf16(v);
        sZ[r * kLdZ + k] = b;
        sb[L::ZT + k * kLdT + warp * kSampW + r] = b;
    }
    __syncwarp();

    // ---- layer 1: h1 = W1z z (tensor cores) + W1u u + b1
    float h1[8][4];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) h1[nb][0] = h1[nb][1] = h1[nb][2] = h1[nb][3] = 0.0f;
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        uint32_t a[4];
        load_a(a, sZ, kLdZ, 0, kb * 16);
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
            uint32_t b[2];
            load_b(b, sb + L::W1z, kLdZ, nb * 8, kb * 16);
            mma16816(h1[nb], a, b);
        }
    }
    const float uxA = wu[2 * g], uyA = wu[2 * g + 1], uxB = wu[2 * (g + 8)], uyB = wu[2 * (g + 8) + 1];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = nb * 8 + 2 * t + (j & 1);
            const float ux = j < 2 ? uxA : uxB, uy = j < 2 ? uyA : uyB;
            h1[nb][j] = h1[nb][j] + sf[L::fW1u + 2 * col] * ux + sf[L::fW1u + 2 * col + 1] * uy + sf[L::fb1 + col];
            const int row = g + (j < 2 ? 0 : 8);
            const __nv_bfloat16 v = to_bf16(silu1(h1[nb][j]));
            sA1[row * kLdH + col] = v;
            sb[L::A1T + col * kLdT + warp * kSampW + row] = v;
        }
    }
    __syncwarp();

    // ---- layer 2 and 3
    float h2[8][4];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) h2[nb][0] = h2[nb][1] = h2[nb][2] = h2[nb][3] = 0.0f;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint32_t a[4];
        load_a(a, sA1, kLdH, 0, kb * 16);
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
            uint32_t b[2];
            load_b(b, sb + L::W2, kLdH, nb * 8, kb * 16);
            mma16816(h2[nb], a, b);
        }
    }
    float yp[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [row A/B][out]
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = nb * 8 + 2 * t + (j & 1);
            h2[nb][j] += sf[L::fb2 + col];
            const float a2 = silu2(h2[nb][j]);
            yp[j >> 1][0] += sf[L::fW3 + col] * a2;
            yp[j >> 1][1] += sf[L::fW3 + kHid + col] * a2;
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            yp[r][o] += __shfl_xor_sync(0xffffffffu, yp[r][o], 1);
            yp[r][o] += __shfl_xor_sync(0xffffffffu, yp[r][o], 2);
            yp[r][o] += sf[L::fb3 + o];
        }
    // ---- loss, outputs, validation
    const int rows[2] = {g, g + 8};
    float dy[2][2];
    float lsum = 0.0f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = rows[r];
        const bool valid = wrc[16 + row] != 0;
        const float ex = yp[r][0] - wu[32 + 2 * row], ey = yp[r][1] - wu[32 + 2 * row + 1];
        dy[r][0] = valid ? 2.0f * ex * A.inv_batch : 0.0f;
        dy[r][1] = valid ? 2.0f * ey * A.inv_batch : 0.0f;
        if (valid && t == 0) {
            lsum += ex * ex + ey * ey;
            if (A.yout) {
                A.yout[2 * (cbase + row)] = yp[r][0];
                A.yout[2 * (cbase + row) + 1] = yp[r][1];
            }
            if (!A.backward && A.val_max_net) {
                const float scv = wu[64 + row];
                const float en = scv * sqrtf(ex * ex + ey * ey);
                const float tx = wu[32 + 2 * row], ty = wu[32 + 2 * row + 1];
                const float es = scv * sqrtf(tx * tx + ty * ty);
                atomicMax(&A.val_max_net[wrc[row]], __float_as_uint(en));
                atomicMax(&A.val_max_series[wrc[row]], __float_as_uint(es));
                atomicAdd(&A.val_sum[0], (double)en);
                atomicAdd(&A.val_sum[1], (double)es);
            }
        }
    }
    for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    float *wg = sf + L::fWG + warp * L::kWG;  // this warp's gradient slots
    if (lane == 0) {
        if (A.backward)
            wg[386] = lsum * A.inv_batch;
        else if (A.loss)
            atomicAdd(A.loss, lsum * A.inv_batch);
    }
    if (!A.backward) return;

    // ---- layer 3 gradients
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = nb * 8 + 2 * t + h;
            float w0 = dy[0][0] * silu2(h2[nb][h]) + dy[1][0] * silu2(h2[nb][2 + h]);
            float w1 = dy[0][1] * silu2(h2[nb][h]) + dy[1][1] * silu2(h2[nb][2 + h]);
            for (int o = 4; o < 32; o <<= 1) {
                w0 += __shfl_xor_sync(0xffffffffu, w0, o);
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
            }
            if (g == 0) {
                wg[col] = w0;
                wg[kHid + col] = w1;
            }
        }
    }
    {
        float d0 = t == 0 ? dy[0][0] + dy[1][0] : 0.0f, d1 = t == 0 ? dy[0][1] + dy[1][1] : 0.0f;
        for (int o = 16; o; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        if (lane == 0) {
            wg[128] = d0;
            wg[129] = d1;
        }
    }
    // ---- dh2 = (dy W3) * silu'(h2)
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = nb * 8 + 2 * t + h;
            float colsum = 0.0f;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float da2 = dy[r][0] * sf[L::fW3 + col] + dy[r][1] * sf[L::fW3 + kHid + col];
                const float d = da2 * dsilu2(h2[nb][2 * r + h]);
                colsum += d;
                const __nv_bfloat16 v = to_bf16(d);
                sDH2[rows[r] * kLdH + col] = v;
                sb[L::DH2T + col * kLdT + warp * kSampW + rows[r]] = v;
            }
            for (int o = 4; o < 32; o <<= 1) colsum += __shfl_xor_sync(0xffffffffu, colsum, o);
            if (g == 0) wg[322 + col] = colsum;
        }
    }
    __syncwarp();
    // ---- da1 = dh2 W2 (tensor cores), dh1 = da1 * silu'(h1)
    float d1[8][4];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) d1[nb][0] = d1[nb][1] = d1[nb][2] = d1[nb][3] = 0.0f;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint32_t a[4];
        load_a(a, sDH2, kLdH, 0, kb * 16);
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
            uint32_t b[2];
            load_b(b, sb + L::W2T, kLdH, nb * 8, kb * 16);
            mma16816(d1[nb], a, b);
        }
    }
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = nb * 8 + 2 * t + h;
            float colsum = 0.0f, gu0 = 0.0f, gu1 = 0.0f;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float d = d1[nb][2 * r + h] * dsilu1(h1[nb][2 * r + h]);
                colsum += d;
                gu0 += d * wu[2 * rows[r]];
                gu1 += d * wu[2 * rows[r] + 1];
                const __nv_bfloat16 v = to_bf16(d);
                sDH1[rows[r] * kLdH + col] = v;
                sb[L::DH1T + col * kLdT + warp * kSampW + rows[r]] = v;
            }
            for (int o = 4; o < 32; o <<= 1) {
                colsum += __shfl_xor_sync(0xffffffffu, colsum, o);
                gu0 += __shfl_xor_sync(0xffffffffu, gu0, o);
                gu1 += __shfl_xor_sync(0xffffffffu, gu1, o);
            }
            if (g == 0) {
                wg[258 + col] = colsum;
                wg[130 + 2 * col] = gu0;
                wg[130 + 2 * col + 1] = gu1;
            }
        }
    }
    __syncwarp();
    // ---- latent gradients dz = dh1 W1z (tensor cores)
    {
        float dzc[4][4];
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) dzc[nb][0] = dzc[nb][1] = dzc[nb][2] = dzc[nb][3] = 0.0f;
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            uint32_t a[4];
            load_a(a, sDH1, kLdH, 0, kb * 16);
#pragma unroll
            for (int nb = 0; nb < 4; ++nb) {
                uint32_t b[2];
                load_b(b, sb + L::W1zT, kLdH, nb * 8, kb * 16);
                mma16816(dzc[nb], a, b);
            }
        }
#pragma unroll
        for (int nb = 0; nb < 4; ++nb) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int row = rows[j >> 1], col = nb * 8 + 2 * t + (j & 1);
                if (!wrc[16 + row]) continue;
                if (expl) {
                    if (A.dzout) A.dzout[(cbase + row) * kLat + col] = dzc[nb][j];
                } else {
                    A.dzs[(cbase + row) * kLat + col] = dzc[nb][j];
                }
            }
        }
    }
    __syncthreads();
    // ---- CTA-level weight gradients over the 128 samples, into this CTA's row
    float *gp = A.gpart + (int64_t)blockIdx.x * kGP;
    {
        // dW2[out][in] = sum_s dh2[s][out] a1[s][in]: warp w takes in-block w
        float c[4][4];
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) c[mb][0] = c[mb][1] = c[mb][2] = c[mb][3] = 0.0f;
#pragma unroll
        for (int kb = 0; kb < kSampC / 16; ++kb) {
            uint32_t b[2];
            load_b(b, sb + L::A1T, kLdT, warp * 8, kb * 16);
#pragma unroll
            for (int mb = 0; mb < 4; ++mb) {
                uint32_t a[4];
                load_a(a, sb + L::DH2T, kLdT, mb * 16, kb * 16);
                mma16816(c[mb], a, b);
            }
        }
#pragma unroll
        for (int mb = 0; mb < 4; ++mb)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int out = mb * 16 + g + (j < 2 ? 0 : 8), in = warp * 8 + 2 * t + (j & 1);
                gp[oW2 + out * kHid + in] = c[mb][j];
            }
    }
    if (warp < 4) {
        // dW1z[out][in] = sum_s dh1[s][out] z[s][in]: warp w takes in-block w
        float c[4][4];
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) c[mb][0] = c[mb][1] = c[mb][2] = c[mb][3] = 0.0f;
#pragma unroll
        for (int kb = 0; kb < kSampC / 16; ++kb) {
            uint32_t b[2];
            load_b(b, sb + L::ZT, kLdT, warp * 8, kb * 16);
#pragma unroll
            for (int mb = 0; mb < 4; ++mb) {
                uint32_t a[4];
                load_a(a, sb + L::DH1T, kLdT, mb * 16, kb * 16);
                mma16816(c[mb], a, b);
            }
        }
#pragma unroll
        for (int mb = 0; mb < 4; ++mb)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int out = mb * 16 + g + (j < 2 ? 0 : 8), in = warp * 8 + 2 * t + (j & 1);
                gp[oW1z + out * kLat + in] = c[mb][j];
            }
    }
    // the per-warp slots, summed over the warps in order
    for (int e = tid; e < 387; e += 256) {
        float acc = 0.0f;
        for (int w = 0; w < 8; ++w) acc += sf[L::fWG + w * L::kWG + e];
        const int dst = e < 128 ? oW3 + e
                      : e < 130 ? ob3 + (e - 128)
                      : e < 258 ? oW1u + (e - 130)
                      : e < 322 ? ob1 + (e - 258)
                      : e < 386 ? ob2 + (e - 322)
                                : kParams;  // the loss
        gp[dst] = acc;
    }
}

cudaError_t ff_train_step(const TrainArgs &t, int64_t nsamples, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_ff_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TrainSmemLayout::bytes);
    if (e != cudaSuccess) return e;
    if (nsamples <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((nsamples + kSampC - 1) / kSampC);
    k_ff_train<<<nb, 256, TrainSmemLayout::bytes, s>>>(t);
    return cudaGetLastError();
}

int64_t ff_gpart_stride() { return kGP; }
int64_t ff_train_blocks(int64_t nsamples) { return (nsamples + kSampC - 1) / kSampC; }

// grads[p] = sum over the CTA rows of gpart in row order (and the loss).
__global__ void k_reduce_grads(const float *__restrict__ gpart, int64_t nblk, float *__restrict__ grads,
                               float *__restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    float acc = 0.0f;
#pragma unroll 8
    for (int64_t b = 0; b < nblk; ++b) acc += gpart[b * kGP + p];
    if (p < kParams)
        grads[p] = acc;
    else if (loss)
        *loss = acc;
}

// dz[c][k] = sum of the step's samples of cell c in sample order: sample li of
// the step is sample offset + li of the sequence, whose cell is its index mod nrc.
__global__ void k_reduce_latents(const float *__restrict__ dzs, int64_t count, int64_t offset, int nrc,
                                 float *__restrict__ dz)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nrc * kLat) return;
    const int c = (int)(e / kLat), k = (int)(e % kLat);
    int64_t li = ((int64_t)c - offset % nrc + nrc) % nrc;
    float acc = 0.0f;
    for (; li < count; li += nrc) acc += dzs[li * kLat + k];
    dz[e] = acc;
}

cudaError_t ff_reduce_grads(const float *gpart, int64_t nblk, float *grads, float *loss, cudaStream_t s)
{
    k_reduce_grads<<<(kParams + 1 + 255) / 256, 256, 0, s>>>(gpart, nblk, grads, loss);
    return cudaGetLastError();
}

cudaError_t ff_reduce_latents(const float *dzs, int64_t count, int64_t offset, int nrc, float *dz, cudaStream_t s)
{
    const int64_t n = (int64_t)nrc * kLat;
    k_reduce_latents<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dzs, count, offset, nrc, dz);
    return cudaGetLastError();
}

__global__ void k_adam(float *p, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

cudaError_t ff_adam(float *p, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                    float bc1, float bc2, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
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
    __align__(128) unsigned char w2cm[kHid * kHid * 2];  // W2 [out][in], BF16, core-matrix layout (B operand)
    uint64_t mbar[2];     // per warpgroup: completion of its tensor-core MMAs
    uint32_t tmem;        // tensor-memory base: 128 columns, 64 per warpgroup
    int wg_ok[8];         // per warp: the last wait completed
    int tc_dead[2];       // per warpgroup: a wait gave up; no more MMAs
    uint32_t pending[2];  // the phase a dead warpgroup still waits for
    float4 l1[kHid];  // per hidden unit: {e_c (this tile's cell), W1u[.][0], W1u[.][1], b2}
    float2 l3[kHid];  // per hidden unit: {W3[0][.], W3[1][.]}
    float b3[2];
    float coef[kCoefStride];
    float sc;
    int rb[3], re[3];
    int nnear;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// One tile of a non-flagged cell: near stars exactly (FP32 recentred + Kahan,
// as the plain kernel), far field = float-pair b0 + series to order pe +
// network residual, then beta and the same binning epilogue.
constexpr int kNearChunk = 8;  // near-field stars per compensated chunk
constexpr int kTcChunk = 128;                            // rays per tensor-core MMA (M)
constexpr int kTcABytes = kTcChunk * kHid * 2;           // one warpgroup's A operand (16 KB)
constexpr int kTcSmem = 2 * kTcABytes;                   // dynamic shared memory of the learned kernel
constexpr int kWaitPolls = 1 << 20;                      // bound on a completion wait

template <bool NET>
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
        float fcx = (float)cxd, fcy = (float)cyd;
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
    if (tid < kHid) ls.l1[tid].x = L.ec ? L.ec[(int64_t)rc * kHid + tid] : 0.0f;
    __syncthreads();

    float2 rx, ry[NP], px[NP], py[NP], Sx[NP], Sy[NP], Cx[NP], Cy[NP];
    const float cxf = ts.tc[0], cyf = ts.tc[1];
    {
        const float kx = (float)tx;
        const float dxr = __fmaf_rn(kx, R.dxh, __fmaf_rn(kx, R.dxl, ts.tc[2]));
        rx = f2(dxr, dxr);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float k0 = (float)(tg * 2 * NP + 2 * p), k1 = k0 + 1.0f;
            ry[p] = f2(__fmaf_rn(k0, R.dyh, __fmaf_rn(k0, R.dyl, ts.tc[3])),
                       __fmaf_rn(k1, R.dyh, __fmaf_rn(k1, R.dyl, ts.tc[3])));
            px[p] = py[p] = Sx[p] = Sy[p] = Cx[p] = Cy[p] = f2(0.f, 0.f);
        }
    }
    // ---- near field: the 3 x 3 block's stars (about 1.3 per tile at the learned
    // workload's density), staged 256 at a time and summed in compensated chunks
    // of kNearChunk stars, padded with massless far stars
    const int nnear = ls.nnear;
    for (int base = 0; base < nnear; base += 256) {
        const int cnt = min(256, nnear - base), cntp = (cnt + kNearChunk - 1) / kNearChunk * kNearChunk;
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
        for (int k0 = 0; k0 < cntp; k0 += kNearChunk) {
#pragma unroll
            for (int k = k0; k < k0 + kNearChunk; ++k) {
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
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                kahan2(Sx[p], Cx[p], px[p]);
                kahan2(Sy[p], Cy[p], py[p]);
                px[p] = py[p] = f2(0.f, 0.f);
            }
        }
    }
    __syncthreads();  // star stages dead; the region now holds the network outputs

    // ---- network residual for the tile's 2048 rays (warp w: rays 256w .. 256w+255)
    float *Y = reinterpret_cast<float *>(sm.hist);
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
        for (int ch = wg; ch < 2048 / kTcChunk; ch += 2) {
            const int r = ch * kTcChunk + t;  // ray of the tile (row-major 64 x 32)
            float y0 = 0.0f, y1 = 0.0f;
            if (!ls.tc_dead[wg]) {
                const float ux = (float)(2 * (ioff + (r & 63)) + 1) * inv_cx - 1.0f;
                const float uy = (float)(2 * (joff + (r >> 6)) + 1) * inv_cy - 1.0f;
#pragma unroll
                for (int k8 = 0; k8 < kHid / 8; ++k8) {
                    uint32_t pk[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c0 = k8 * 8 + 2 * q;
                        const float4 p0 = ls.l1[c0], p1 = ls.l1[c0 + 1];
                        const float v0 = silu1(p0.x + p0.y * ux + p0.z * uy);
                        const float v1 = silu1(p1.x + p1.y * ux + p1.z * uy);
                        pk[q] = pack_bf16(v0, v1);
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
                const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&ls.mbar[wg], phase, kWaitPolls));
                if (lane == 0) ls.wg_ok[warp] = ok ? 1 : 0;
                umma::wg_sync(wg);
                const bool wg_ok = ls.wg_ok[4 * wg] && ls.wg_ok[4 * wg + 1] && ls.wg_ok[4 * wg + 2] &&
                                   ls.wg_ok[4 * wg + 3];
                if (wg_ok) {
                    phase ^= 1u;
                    umma::fence_after();
#pragma unroll
                    for (int c0 = 0; c0 < kHid; c0 += 16) {
                        uint32_t acc[16];
                        umma::ld16(dcol + lane_base + (uint32_t)c0, acc);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int col = c0 + j;
                            const float a2 = silu2(__uint_as_float(acc[j]) + ls.l1[col].w);
                            const float2 w3 = ls.l3[col];
                            y0 += w3.x * a2;
                            y1 += w3.y * a2;
                        }
                    }
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
            Y[2 * r] = y0 + ls.b3[0];
            Y[2 * r + 1] = y1 + ls.b3[1];
        }
    }
    __syncthreads();

    // ---- far field and beta per ray
    float bxh[2 * NP], byh[2 * NP], bxl[2 * NP], byl[2 * NP];
    const float uxr = (float)(2 * (ioff + tx) + 1) * inv_cx - 1.0f;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 2 * p + h;
            const int jl = tg * 2 * NP + r;
            const float uyr = (float)(2 * (joff + jl) + 1) * inv_cy - 1.0f;
            const float2 v = make_float2(uxr * 0.70710678f, uyr * 0.70710678f);
            // T = sum_{p=1}^{pe} b_p v^p + v^(pe+1) q, q = s_c (network output) or 0:
            // Horner with q as the innermost coefficient
            float2 acc = make_float2(0.f, 0.f);
            if (L.use_net) {
                const int ray = jl * kTileX + tx;
                acc = make_float2(ls.sc * Y[2 * ray], ls.sc * Y[2 * ray + 1]);
            }
            acc = cmul(acc, v);
            for (int q = L.pe; q >= 1; --q) {
                acc.x += ls.coef[4 + 2 * (q - 1)];
                acc.y += ls.coef[5 + 2 * (q - 1)];
                acc = cmul(acc, v);
            }
            const float rx_ = 0.f, ry_ = 0.f;
            const float sx = h ? Sx[p].y : Sx[p].x, sy = h ? Sy[p].y : Sy[p].x;
            const float ccx = h ? Cx[p].y : Cx[p].x, ccy = h ? Cy[p].y : Cy[p].x;
            const float dxr = rx.x, dyr = h ? ry[p].y : ry[p].x;
            const float lx = __fmaf_rn(a.lens.fa11, dxr, __fmul_rn(a.lens.fa12, dyr));
            const float ly = __fmaf_rn(a.lens.fa12, dxr, __fmul_rn(a.lens.fa22, dyr));
            // alpha_far = (Re F, -Im F) + residual;  F = b0 + T
            float th, tl, t2;
            two_sum(ts.tc[4], -sx, th, tl);
            two_sum(th, -ls.coef[0], th, t2);
            float small = __fadd_rn(__fadd_rn(ts.tc[6], ccx), lx);
            small = __fsub_rn(small, __fadd_rn(__fadd_rn(ls.coef[2], acc.x), rx_));
            tl = __fadd_rn(__fadd_rn(tl, t2), small);
            two_sum(th, tl, bxh[r], bxl[r]);
            two_sum(ts.tc[5], -sy, th, tl);
            two_sum(th, ls.coef[1], th, t2);
            small = __fadd_rn(__fadd_rn(ts.tc[7], ccy), ly);
            small = __fadd_rn(small, __fsub_rn(__fadd_rn(ls.coef[3], acc.y), ry_));
            tl = __fadd_rn(__fadd_rn(tl, t2), small);
            two_sum(th, tl, byh[r], byl[r]);
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

// NET: the network on the tensor cores (tcgen05; tensor memory and kTcSmem bytes
// of dynamic shared memory); without it (the series alone) the kernel carries no
// tensor-core code and no dynamic shared memory.
template <int NRP, bool NET>
__global__ void __launch_bounds__(kThreads, 2) k_shoot_learned(LearnedArgs L)
{
    __shared__ __align__(16) ShootSmem<256> sm;
    __shared__ TileShared ts;
    __shared__ __align__(128) LearnSmem ls;
    __shared__ long long s_item;
    extern __shared__ __align__(128) unsigned char tc_abuf[];  // two A operands, kTcSmem bytes
    const int tid = threadIdx.x;
    uint32_t phase = 0;  // completed MMA batches of this thread's warpgroup, mod 2
    if (NET) {
        for (int i = tid; i < kHid * kHid; i += kThreads)
            *reinterpret_cast<__nv_bfloat16 *>(ls.w2cm + umma::cm_offset(i / kHid, i % kHid)) = L.w2b[i];
        if (tid < kHid) {
            ls.l1[tid].y = L.params[oW1u + 2 * tid];
            ls.l1[tid].z = L.params[oW1u + 2 * tid + 1];
            ls.l1[tid].w = L.params[ob2 + tid];
            ls.l3[tid] = make_float2(L.params[oW3 + tid], L.params[oW3 + kHid + tid]);
        }
        if (tid < 2) ls.b3[tid] = L.params[ob3 + tid];
        if (tid < 2) ls.tc_dead[tid] = 0;
        if (tid == 0) {
            umma::mbar_init(&ls.mbar[0], 1);
            umma::mbar_init(&ls.mbar[1], 1);
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
            shoot_tile<4, 256, false, NRP>(L.plain, bx, by, sm, ts);
        else
            learned_tile<NET>(L, bx, by, sm, ts, ls, tc_abuf, phase);
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
// carveout for two CTAs of ~59 KB per SM.
template <class K>
static cudaError_t learned_attributes(K kernel)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t ff_learned_grid(int *grid)
{
    // The persistent grid takes the resident CTAs per SM of the kernel without
    // tensor-core code (two: registers, launch-bounded to 128 per thread).  The
    // tensor-core variant has the same register and shared-memory limits (ncu: 2
    // by registers, 3 by shared memory), though the occupancy query reports one
    // for it; CTAs beyond those resident only find the shared work queue empty.
    int per_sm = 0, per_sm1 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shoot_learned<0, false>, kThreads, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, k_shoot_learned<1, false>, kThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < per_sm1 ? per_sm : per_sm1;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *grid = nsm * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

template <int NRP>
static cudaError_t launch_learned(const LearnedArgs &L, unsigned g, cudaStream_t s)
{
    if (L.use_net) {
        cudaError_t e = learned_attributes(k_shoot_learned<NRP, true>);
        if (e != cudaSuccess) return e;
        k_shoot_learned<NRP, true><<<g, kThreads, kTcSmem, s>>>(L);
    } else {
        k_shoot_learned<NRP, false><<<g, kThreads, 0, s>>>(L);
    }
    return cudaGetLastError();
}

cudaError_t ff_shoot_learned(const LearnedArgs &L, int grid, int fma_pairs, cudaStream_t s)
{
    const int64_t g = L.nitems < grid ? (L.nitems > 0 ? L.nitems : 1) : grid;
    return fma_pairs ? launch_learned<1>(L, (unsigned)g, s) : launch_learned<0>(L, (unsigned)g, s);
}

}  // namespace mlens
