// lightcurve.cu -- the magnification map convolved with a source's intensity
// profile, and light curves sampled from it (Section 1: given a model of the
// background source's size and intensity profile, the magnification pattern
// yields simulated light curves).  Declared in include/mlens.h.
//
//   out[j][i] = scale * sum_{(di,dj) in K} w(di,dj) counts[j+dj][i+di],
//   counts = 0 outside the map, weights normalised to sum 1 over K.
//
// Gaussian profile: separable, so two HBM-bound passes over the map -- rows
// (uint32 counts -> FP32) and columns (FP32 -> FP32 x scale) -- each staging a
// tile plus its halo in shared memory and taking every tap from there.
// Uniform disk: each row of the disk's support is one contiguous run of pixels,
// so with per-row inclusive prefix sums P (int64, exact) an output is
// sum over the support's rows of P[row][i+h] - P[row][i-h-1]: O(rows) work per
// pixel, exact integer sums, then (float)(sum * (scale / |K|)) in FP64.
// Light curve: bilinear interpolation between pixel centres along a straight
// source track, in FP64 with explicit round-to-nearest operations.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "mlens_internal.h"

namespace mlens {
namespace {

constexpr int kThr = 256;
constexpr int kRowOut = 1024;   // row pass: outputs per CTA
constexpr int kColX = 64;       // column pass: tile columns
constexpr int kColY = 128;      // column pass: tile rows
constexpr int kMaxTaps = 256;   // Gaussian half-width limit (pixels)
constexpr int kMaxDiskRows = 4096;

__host__ __device__ constexpr int taps_padded(int K) { return (2 * K + 1 + 3) / 4 * 4; }

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Row pass.  A CTA takes kRowOut outputs of two adjacent rows; thread t computes
// the four consecutive outputs 4t .. 4t+3 of both rows, the rows packed into the
// two lanes of f32x2 registers (FFMA2), with a sliding window stepped four taps
// at a time: per four taps two float4 loads of duplicated weights (broadcast),
// four float2 input loads and sixteen FFMA2 = 32 multiply-adds.  Each output
// takes its taps in the same order as a scalar loop would: the packing changes
// no result.  The weights are zero-padded to a multiple of four (adding exact
// zeros).  The staged inputs are stored de-interleaved by index mod 4 (plane
// e % 4, slot e / 4) so that the lanes' loads of element 4t + k are consecutive.
__global__ void __launch_bounds__(kThr) k_gauss_rows(const uint32_t *__restrict__ in, int nx, int ny,
                                                     const float *__restrict__ w, int K, float *__restrict__ out)
{
    extern __shared__ float4 sm4[];
    const int Kp = taps_padded(K);
    float2 *ws = reinterpret_cast<float2 *>(sm4);  // Kp weights, each duplicated (w, w)
    const int E = kRowOut + Kp + 3;                // staged inputs per row
    const int P = E / 4 + 1;
    float2 *xs = ws + Kp;                          // 4 planes of P (row j, row j + 1) pairs
    const int tid = threadIdx.x;
    for (int k = tid; k < Kp; k += kThr) {
        const float v = k <= 2 * K ? w[k] : 0.0f;
        ws[k] = make_float2(v, v);
    }
    const int i0 = blockIdx.x * kRowOut;
    const int o = 4 * tid;  // this thread's first output within the tile
    for (int64_t j = 2 * (int64_t)blockIdx.y; j < ny; j += 2 * (int64_t)gridDim.y) {
        const bool two = j + 1 < ny;
        const uint32_t *row0 = in + j * nx, *row1 = row0 + nx;
        __syncthreads();  // previous rows' taps are done
        for (int e = tid; e < E; e += kThr) {
            const int i = i0 - K + e;
            const bool inside = i >= 0 && i < nx;
            xs[(e & 3) * P + (e >> 2)] =
                make_float2(inside ? (float)row0[i] : 0.0f, inside && two ? (float)row1[i] : 0.0f);
        }
        __syncthreads();
        if (i0 + o < nx) {
            // element 4t + 4m + d sits in plane d & 3, slot t + m + (d >> 2)
            const float2 *b = xs + tid;
            const float4 *wq = sm4;  // (w_2n, w_2n, w_2n+1, w_2n+1)
            float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
            float2 x0 = b[0], x1 = b[P], x2 = b[2 * P];
            // (unrolled so that the next steps' loads issue ahead of this step's FFMA2s)
#pragma unroll 8
            for (int m = 0; m < Kp / 4; ++m) {
                const float4 qa = wq[2 * m], qb = wq[2 * m + 1];
                const float2 w0 = make_float2(qa.x, qa.y), w1 = make_float2(qa.z, qa.w);
                const float2 w2 = make_float2(qb.x, qb.y), w3 = make_float2(qb.z, qb.w);
                const float2 x3 = b[3 * P + m], x4 = b[m + 1], x5 = b[P + m + 1], x6 = b[2 * P + m + 1];
                a0 = ffma2(w0, x0, a0); a1 = ffma2(w0, x1, a1); a2 = ffma2(w0, x2, a2); a3 = ffma2(w0, x3, a3);
                a0 = ffma2(w1, x1, a0); a1 = ffma2(w1, x2, a1); a2 = ffma2(w1, x3, a2); a3 = ffma2(w1, x4, a3);
                a0 = ffma2(w2, x2, a0); a1 = ffma2(w2, x3, a1); a2 = ffma2(w2, x4, a2); a3 = ffma2(w2, x5, a3);
                a0 = ffma2(w3, x3, a0); a1 = ffma2(w3, x4, a1); a2 = ffma2(w3, x5, a2); a3 = ffma2(w3, x6, a3);
                x0 = x4;
                x1 = x5;
                x2 = x6;
            }
            const int n = min(4, nx - (i0 + o));
            float *orow = out + j * nx + i0 + o;
            orow[0] = a0.x;
            if (n > 1) orow[1] = a1.x;
            if (n > 2) orow[2] = a2.x;
            if (n > 3) orow[3] = a3.x;
            if (two) {
                orow += nx;
                orow[0] = a0.y;
                if (n > 1) orow[1] = a1.y;
                if (n > 2) orow[2] = a2.y;
                if (n > 3) orow[3] = a3.y;
            }
        }
    }
}

// Column pass.  A CTA stages kColY + Kp + 3 rows of 64 columns; thread (p, g)
// computes rows 16g .. 16g+15 of the adjacent columns 2p and 2p + 1 (packed into
// f32x2 lanes) in blocks of eight consecutive rows, with the same four-taps-at-a-
// time window (the lanes of a warp read 32 consecutive column pairs of one staged
// row).  As in the row pass, every output's taps keep their order.
__global__ void __launch_bounds__(kThr) k_gauss_cols(const float *__restrict__ in, int nx, int ny,
                                                     const float *__restrict__ w, int K, float scale,
                                                     float *__restrict__ out)
{
    extern __shared__ float4 sm4[];
    const int Kp = taps_padded(K);
    float2 *ws = reinterpret_cast<float2 *>(sm4);        // Kp weights, each duplicated (w, w)
    float *tile = reinterpret_cast<float *>(ws + Kp);    // (kColY + Kp + 3) rows x kColX columns
    const int tid = threadIdx.x;
    for (int k = tid; k < Kp; k += kThr) {
        const float v = k <= 2 * K ? w[k] : 0.0f;
        ws[k] = make_float2(v, v);
    }
    const int lc = tid % kColX, lg = tid / kColX;        // staging: column, row group
    const int cp = tid % (kColX / 2), g = tid / (kColX / 2);  // compute: column pair, group of kColY / 8 rows
    const int il = blockIdx.x * kColX + lc;
    const int i = blockIdx.x * kColX + 2 * cp;           // first column of this thread's pair
    const int rows = kColY + Kp + 3;
    const int tiles_y = (ny + kColY - 1) / kColY;
    for (int ty = blockIdx.y; ty < tiles_y; ty += gridDim.y) {
        const int64_t j0 = (int64_t)ty * kColY;
        __syncthreads();
        for (int r = lg; r < rows; r += kThr / kColX) {
            const int64_t j = j0 - K + r;
            tile[r * kColX + lc] = (il < nx && j >= 0 && j < ny) ? in[j * nx + il] : 0.0f;
        }
        __syncthreads();
        if (i >= nx) continue;
        const bool two = i + 1 < nx;
        for (int r = g * (kColY / 8); r < (g + 1) * (kColY / 8); r += 8) {
            if (j0 + r >= ny) break;
            const float2 *T = reinterpret_cast<const float2 *>(tile + r * kColX + 2 * cp);
            constexpr int S = kColX / 2;  // float2 per staged row
            float2 a[8], x[11];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 7; ++q) x[q] = T[q * S];
#pragma unroll 4
            for (int k = 0; k < Kp; k += 4) {
                const float4 qa = sm4[k >> 1], qb = sm4[(k >> 1) + 1];
                const float2 w0 = make_float2(qa.x, qa.y), w1 = make_float2(qa.z, qa.w);
                const float2 w2 = make_float2(qb.x, qb.y), w3 = make_float2(qb.z, qb.w);
#pragma unroll
                for (int q = 0; q < 4; ++q) x[7 + q] = T[(k + 7 + q) * S];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    a[q] = ffma2(w0, x[q], a[q]);
                    a[q] = ffma2(w1, x[q + 1], a[q]);
                    a[q] = ffma2(w2, x[q + 2], a[q]);
                    a[q] = ffma2(w3, x[q + 3], a[q]);
                }
#pragma unroll
                for (int q = 0; q < 7; ++q) x[q] = x[q + 4];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (j0 + r + q < ny) {
                    float *dst = out + (j0 + r + q) * nx + i;
                    dst[0] = __fmul_rn(a[q].x, scale);
                    if (two) dst[1] = __fmul_rn(a[q].y, scale);
                }
        }
    }
}

// Inclusive prefix sums of each row (int64): one CTA per row, 8 elements per thread
// per chunk, warp shuffles then one shared-memory step across the 8 warps.  A
// chunk's counts are read, and its sums written, through shared memory so that
// the global accesses are coalesced (a thread's own 8 elements are consecutive).
__global__ void __launch_bounds__(kThr) k_row_prefix(const uint32_t *__restrict__ in, int nx, int ny,
                                                     int64_t *__restrict__ P)
{
    constexpr int kPer = 8, kChunk = kThr * kPer;
    __shared__ int64_t wsum[kThr / 32];
    __shared__ int64_t carry_s;
    __shared__ __align__(16) uint32_t cin[kChunk];
    __shared__ __align__(16) int64_t cout[kChunk + kChunk / kPer];  // element e at e + e / 8: no bank conflicts
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t j = blockIdx.x; j < ny; j += gridDim.x) {
        const uint32_t *row = in + j * nx;
        int64_t *prow = P + j * nx;
        int64_t carry = 0;
        for (int64_t base = 0; base < nx; base += kChunk) {
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int64_t i = base + k * kThr + tid;
                cin[k * kThr + tid] = i < nx ? row[i] : 0u;
            }
            __syncthreads();
            const uint4 c0 = reinterpret_cast<const uint4 *>(cin)[2 * tid];
            const uint4 c1 = reinterpret_cast<const uint4 *>(cin)[2 * tid + 1];
            const uint32_t cv[kPer] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            int64_t v[kPer];
            int64_t run = 0;
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                run += (int64_t)cv[k];  // zero past the row's end
                v[k] = run;
            }
            int64_t x = run;  // inclusive scan of the thread totals across the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            int64_t before = 0;
            for (int q = 0; q < warp; ++q) before += wsum[q];
            const int64_t off = carry + before + (x - run);
#pragma unroll
            for (int k = 0; k < kPer; ++k) cout[tid * (kPer + 1) + k] = off + v[k];
            if (tid == kThr - 1) carry_s = off + run;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int64_t i = base + k * kThr + tid;
                const int e = k * kThr + tid;
                if (i < nx) prow[i] = cout[e + e / kPer];
            }
            carry = carry_s;
            __syncthreads();  // wsum, carry_s, cin and cout are reused by the next chunk
        }
    }
}

__global__ void __launch_bounds__(kThr) k_disk(const int64_t *__restrict__ P, int nx, int ny,
                                               const int *__restrict__ half, int H, double f,
                                               float *__restrict__ out)
{
    extern __shared__ int hs[];  // 2H+1 half-widths
    const int tid = threadIdx.x;
    for (int k = tid; k <= 2 * H; k += kThr) hs[k] = half[k];
    __syncthreads();
    const int i = blockIdx.x * kThr + tid;
    for (int64_t j = blockIdx.y; j < ny; j += gridDim.y) {
        if (i >= nx) continue;
        int64_t s = 0;
        for (int d = -H; d <= H; ++d) {
            const int64_t jj = j + d;
            if (jj < 0 || jj >= ny) continue;
            const int h = hs[d + H];
            const int64_t *pr = P + jj * nx;
            const int hi = min(i + h, nx - 1);
            const int lo = i - h - 1;
            s += pr[hi] - (lo >= 0 ? pr[lo] : 0);
        }
        out[j * nx + i] = __double2float_rn(__dmul_rn((double)s, f));
    }
}

// The same sums for disks of moderate size, with the prefix sums a tile needs staged
// in shared memory once: a CTA takes kDiskTX x kDiskTY outputs and loads rows
// j0 - H .. j0 + kDiskTY - 1 + H, columns i0 - W - 1 .. i0 + kDiskTX - 1 + W of P
// (W: the largest half-width), with 0 above and below the map and left of it and
// P[row][nx - 1] right of it -- exactly the values k_disk's clamps produce, so the
// integer sums, and the outputs, are identical.  The 2 (2H + 1) loads per output
// then come from shared memory instead of L2.  Thread (c, g) computes column c of
// rows 8 g .. 8 g + 7 of the tile.
constexpr int kDiskTX = 64, kDiskTY = 32;

// 8-byte asynchronous global -> shared copy (Ampere-style cp.async: no register round
// trip, so all of a thread's copies are in flight at once); n = 0 writes zeros and
// reads nothing.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int n)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
constexpr size_t kDiskTileMaxSmem = 100 * 1024;  // above this the plain kernel runs

__host__ __device__ constexpr size_t disk_tile_smem(int H, int W)
{
    return ((size_t)kDiskTY + 2 * (size_t)H) * ((size_t)kDiskTX + 2 * (size_t)W + 1) * sizeof(int64_t) +
           (2 * (size_t)H + 1) * sizeof(int);  // size_t throughout: W can be as large as nx
}

__global__ void __launch_bounds__(kThr) k_disk_tile(const int64_t *__restrict__ P, int nx, int ny,
                                                    const int *__restrict__ half, int H, int W, double f,
                                                    float *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int rows = kDiskTY + 2 * H, cols = kDiskTX + 2 * W + 1;
    int64_t *T = reinterpret_cast<int64_t *>(dsm);
    int *hs = reinterpret_cast<int *>(T + (size_t)rows * cols);
    const int tid = threadIdx.x, c = tid % kDiskTX, g = tid / kDiskTX;
    const int i0 = blockIdx.x * kDiskTX;
    for (int k = tid; k <= 2 * H; k += kThr) hs[k] = min(half[k], W);  // half[k] <= W: a guard only
    const int64_t tiles_y = ((int64_t)ny + kDiskTY - 1) / kDiskTY;
    for (int64_t by = blockIdx.y; by < tiles_y; by += gridDim.y) {
        const int64_t j0 = by * kDiskTY, jbase = j0 - H;
        const int64_t cbase = (int64_t)i0 - W - 1;
        __syncthreads();  // the previous tile's reads are done
        for (int r = tid / 32; r < rows; r += kThr / 32) {  // a warp per row, its lanes along it
            const int64_t jj = jbase + r;
            const bool in = jj >= 0 && jj < ny;
            for (int q = tid % 32; q < cols; q += 32) {
                const int64_t col = cbase + q;
                const bool ok = in && col >= 0;
                cp_async8(&T[r * cols + q], ok ? P + jj * nx + (col < nx ? col : nx - 1) : P, ok ? 8 : 0);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        const int i = i0 + c;
        if (i < nx) {
            constexpr int kRows = kDiskTY / 4;  // output rows per thread
            const int rt0 = g * kRows;          // the thread's first row within the tile
            int64_t sum[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) sum[k] = 0;
            // T row rt0 + d is row j0 + rt0 - H + d of the map; tr[0] is the column of i - 1.
            // rs[k]: the run sum of output k at support row d.  Where the next support row
            // has the same half-width (a warp-uniform test), output k's next run is output
            // k + 1's current one, so the runs shift by one and only the last is loaded.
            const int64_t *tr = T + (size_t)rt0 * cols + c + W;
            int64_t rs[kRows];
            int hprev = -1;
            for (int d = 0; d <= 2 * H; ++d) {  // one half-width per support row, for all kRows outputs
                const int h = hs[d];
                if (h == hprev) {
#pragma unroll
                    for (int k = 0; k < kRows - 1; ++k) rs[k] = rs[k + 1];
                    rs[kRows - 1] = tr[(kRows - 1) * cols + h + 1] - tr[(kRows - 1) * cols - h];
                } else {
#pragma unroll
                    for (int k = 0; k < kRows; ++k) rs[k] = tr[k * cols + h + 1] - tr[k * cols - h];
                }
#pragma unroll
                for (int k = 0; k < kRows; ++k) sum[k] += rs[k];
                hprev = h;
                tr += cols;
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int64_t j = j0 + rt0 + k;
                if (j < ny) out[j * nx + i] = __double2float_rn(__dmul_rn((double)sum[k], f));
            }
        }
    }
}

// Normalised 1-D Gaussian weights exp(-((k-K) d)^2 / (2 sigma^2)) / sum, one CTA:
// FP64 terms, a fixed-order tree sum, float results.
__global__ void __launch_bounds__(kThr) k_gauss_weights(double sigma, double d, int K, float *__restrict__ w)
{
    __shared__ double e[2 * kMaxTaps + 1];
    __shared__ double part[kThr];
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int k = tid; k <= 2 * K; k += kThr) {
        const double off = __dmul_rn((double)(k - K), d);
        e[k] = exp(-__ddiv_rn(__dmul_rn(off, off), __dmul_rn(2.0, __dmul_rn(sigma, sigma))));
        acc = __dadd_rn(acc, e[k]);
    }
    part[tid] = acc;
    __syncthreads();
    for (int h = kThr / 2; h > 0; h >>= 1) {
        if (tid < h) part[tid] = __dadd_rn(part[tid], part[tid + h]);
        __syncthreads();
    }
    const double sum = part[0];
    for (int k = tid; k <= 2 * K; k += kThr) w[k] = __double2float_rn(__ddiv_rn(e[k], sum));
}

// Half-width of each row dj = q - H of the disk support: the largest h with
// (h dx)^2 + (dj dy)^2 <= R^2 in FP64 without contraction (the definition of the
// support), capped at nx (a longer run changes nothing: both ends clamp).
__global__ void __launch_bounds__(kThr) k_disk_halves(double R, double dx, double dy, int H, int nx,
                                                      int *__restrict__ half)
{
    const int q = blockIdx.x * kThr + threadIdx.x;
    if (q > 2 * H) return;
    const double dj = (double)(q - H);
    const double yy = __dmul_rn(__dmul_rn(dj, dy), __dmul_rn(dj, dy));
    const double rr = __dmul_rn(R, R);
    auto inside = [&](long long h) {
        const double x = __dmul_rn((double)h, dx);
        return __dadd_rn(__dmul_rn(x, x), yy) <= rr;
    };
    long long h = (long long)floor(__ddiv_rn(__dsqrt_rn(fmax(__dsub_rn(rr, yy), 0.0)), dx));
    while (h > 0 && !inside(h)) --h;
    while (h < nx && inside(h + 1)) ++h;
    half[q] = (int)min(h, (long long)nx);
}

struct Track {
    double x0, y0, dx, dy;      // map origin and pixel widths
    double bx0, by0, bx1, by1;  // track end points
    int nx, ny, n;
};

__global__ void __launch_bounds__(kThr) k_curve(const float *__restrict__ m, Track T, float *__restrict__ out)
{
    const int k = blockIdx.x * kThr + threadIdx.x;
    if (k >= T.n) return;
    const double t = T.n > 1 ? __ddiv_rn((double)k, (double)(T.n - 1)) : 0.0;
    const double bx = __dadd_rn(T.bx0, __dmul_rn(t, __dsub_rn(T.bx1, T.bx0)));
    const double by = __dadd_rn(T.by0, __dmul_rn(t, __dsub_rn(T.by1, T.by0)));
    const double u = __dsub_rn(__ddiv_rn(__dsub_rn(bx, T.x0), T.dx), 0.5);
    const double v = __dsub_rn(__ddiv_rn(__dsub_rn(by, T.y0), T.dy), 0.5);
    const double fi = floor(u), fj = floor(v);
    const double fx = __dsub_rn(u, fi), fy = __dsub_rn(v, fj);
    // corner indices clamped before the conversion (only the map's edges matter)
    const int i0 = (int)fmin(fmax(fi, -2.0), (double)T.nx + 1.0);
    const int j0 = (int)fmin(fmax(fj, -2.0), (double)T.ny + 1.0);
    const int ia = min(max(i0, 0), T.nx - 1), ib = min(max(i0 + 1, 0), T.nx - 1);
    const int ja = min(max(j0, 0), T.ny - 1), jb = min(max(j0 + 1, 0), T.ny - 1);
    const double m00 = m[(int64_t)ja * T.nx + ia], m01 = m[(int64_t)ja * T.nx + ib];
    const double m10 = m[(int64_t)jb * T.nx + ia], m11 = m[(int64_t)jb * T.nx + ib];
    const double gx = __dsub_rn(1.0, fx), gy = __dsub_rn(1.0, fy);
    const double s0 = __dadd_rn(__dmul_rn(gx, m00), __dmul_rn(fx, m01));
    const double s1 = __dadd_rn(__dmul_rn(gx, m10), __dmul_rn(fx, m11));
    out[k] = __double2float_rn(__dadd_rn(__dmul_rn(gy, s0), __dmul_rn(fy, s1)));
}

int lc_cuda(cudaError_t e, const char *what)
{
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    clear_pending_error();
    return e == cudaErrorMemoryAllocation ? MLENS_ERR_NOMEM : MLENS_ERR_CUDA;
}

int lc_fail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

int check_map(const mlens_grid *g)
{
    if (!g) return lc_fail(MLENS_ERR_ARG, "source grid is NULL");
    if (!std::isfinite(g->x0) || !std::isfinite(g->x1) || !std::isfinite(g->y0) || !std::isfinite(g->y1) ||
        !(g->x1 > g->x0) || !(g->y1 > g->y0))
        return lc_fail(MLENS_ERR_ARG, "source box must be finite with x1 > x0 and y1 > y0");
    if (g->nx < 1 || g->ny < 1 || (int64_t)g->nx * g->ny > (int64_t(1) << 30))
        return lc_fail(MLENS_ERR_ARG, "source map needs nx, ny >= 1 and nx*ny <= 2^30");
    return MLENS_OK;
}

// Largest di >= 0 with (di dx)^2 + (dj dy)^2 <= R^2, or -1 if none (FP64, as the
// definition of the support).
int half_width(double R, double dx, double dy, int dj)
{
    const double yy = ((double)dj * dy) * ((double)dj * dy);
    if (yy > R * R) return -1;
    auto inside = [&](int64_t h) { return ((double)h * dx) * ((double)h * dx) + yy <= R * R; };
    int64_t h = (int64_t)std::floor(std::sqrt(R * R - yy) / dx);  // within a step or two of the answer
    while (h > 0 && !inside(h)) --h;
    while (inside(h + 1)) ++h;
    return (int)h;
}

}  // namespace
}  // namespace mlens

using namespace mlens;

namespace mlens {
namespace {

// Shape of one convolution: taps / support rows and the workspace layout.
struct ConvPlan {
    int Kx = 0, Ky = 0;    // Gaussian half-widths (pixels)
    int Hs = 0;            // disk: support rows |dj| <= Hs
    int Ws = 0;            // disk: the largest half-width, capped at nx
    int64_t count = 0;     // disk: |K|
    size_t off_map = 0;    // workspace offset of the map-sized buffer
    size_t bytes = 0;      // workspace size
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int plan_convolution(const mlens_grid *src, int32_t profile, double size, ConvPlan *pl)
{
    int rc;
    if ((rc = check_map(src))) return rc;
    if (!std::isfinite(size) || size < 0.0) return lc_fail(MLENS_ERR_ARG, "size must be finite and >= 0");
    const int nx = src->nx, ny = src->ny;
    const size_t npix = (size_t)nx * (size_t)ny;
    const double dx = (src->x1 - src->x0) / nx, dy = (src->y1 - src->y0) / ny;
    if (profile == MLENS_PROFILE_GAUSSIAN) {
        if (!(size > 0.0)) return lc_fail(MLENS_ERR_ARG, "a Gaussian profile needs size > 0");
        if (4.0 * size / dx > kMaxTaps || 4.0 * size / dy > kMaxTaps)
            return lc_fail(MLENS_ERR_ARG, "Gaussian profile wider than 4 sigma = 256 pixels");
        pl->Kx = (int)std::ceil(4.0 * size / dx);
        pl->Ky = (int)std::ceil(4.0 * size / dy);
        pl->off_map = round256((size_t)(2 * pl->Kx + 1 + 2 * pl->Ky + 1) * sizeof(float));
        pl->bytes = pl->off_map + round256(npix * sizeof(float));
        return MLENS_OK;
    }
    if (profile == MLENS_PROFILE_DISK) {
        const int H = (int)std::floor(size / dy) + 1;
        if (H > kMaxDiskRows) return lc_fail(MLENS_ERR_ARG, "disk profile taller than 4096 pixels");
        if (size / dx > 1e9) return lc_fail(MLENS_ERR_ARG, "disk profile wider than 1e9 pixels");
        int64_t count = 0;
        int Hs = 0;
        for (int dj = -H; dj <= H; ++dj) {
            const int h = half_width(size, dx, dy, dj);
            if (h >= 0) {
                count += 2 * (int64_t)h + 1;
                Hs = std::max(Hs, std::abs(dj));
                pl->Ws = std::max(pl->Ws, std::min(h, nx));
            }
        }
        pl->Hs = Hs;
        pl->count = count;
        pl->off_map = round256((size_t)(2 * Hs + 1) * sizeof(int));
        pl->bytes = pl->off_map + round256(npix * sizeof(int64_t));
        return MLENS_OK;
    }
    return lc_fail(MLENS_ERR_ARG, "unknown profile");
}

int run_convolution(const uint32_t *counts_dev, const mlens_grid *src, int32_t profile, double size, double scale,
                    float *out_dev, const ConvPlan &pl, char *work, cudaStream_t s)
{
    const int nx = src->nx, ny = src->ny;
    const double dx = (src->x1 - src->x0) / nx, dy = (src->y1 - src->y0) / ny;
    cudaError_t e;
    if (profile == MLENS_PROFILE_GAUSSIAN) {
        float *wx = reinterpret_cast<float *>(work), *wy = wx + (2 * pl.Kx + 1);
        float *t = reinterpret_cast<float *>(work + pl.off_map);
        k_gauss_weights<<<1, kThr, 0, s>>>(size, dx, pl.Kx, wx);
        k_gauss_weights<<<1, kThr, 0, s>>>(size, dy, pl.Ky, wy);
        if ((e = cudaGetLastError()) != cudaSuccess) return lc_cuda(e, "weights launch");
        const int kpx = taps_padded(pl.Kx), kpy = taps_padded(pl.Ky);
        const size_t sm_r = (size_t)(kpx + 4 * ((kRowOut + kpx + 3) / 4 + 1)) * sizeof(float2);
        const size_t sm_c = (size_t)(2 * kpy + (kColY + kpy + 3) * kColX) * sizeof(float);
        if ((e = cudaFuncSetAttribute(k_gauss_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_r)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k_gauss_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_c)) !=
                cudaSuccess)
            return lc_cuda(e, "cudaFuncSetAttribute");
        const dim3 gr((unsigned)((nx + kRowOut - 1) / kRowOut), (unsigned)std::min<int64_t>((ny + 1) / 2, 65535));
        k_gauss_rows<<<gr, kThr, sm_r, s>>>(counts_dev, nx, ny, wx, pl.Kx, t);
        if ((e = cudaGetLastError()) != cudaSuccess) return lc_cuda(e, "row pass launch");
        const int64_t tiles_y = (ny + kColY - 1) / kColY;
        const dim3 gc((unsigned)((nx + kColX - 1) / kColX), (unsigned)std::min<int64_t>(tiles_y, 65535));
        k_gauss_cols<<<gc, kThr, sm_c, s>>>(t, nx, ny, wy, pl.Ky, (float)scale, out_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return lc_cuda(e, "column pass launch");
        return MLENS_OK;
    }
    int *half = reinterpret_cast<int *>(work);
    int64_t *P = reinterpret_cast<int64_t *>(work + pl.off_map);
    int dev = 0, nsm = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return lc_cuda(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return lc_cuda(e, "cudaDeviceGetAttribute");
    k_disk_halves<<<(unsigned)((2 * pl.Hs + 1 + kThr - 1) / kThr), kThr, 0, s>>>(size, dx, dy, pl.Hs, nx, half);
    const unsigned gp = (unsigned)std::min<int64_t>(ny, (int64_t)nsm * 8);
    k_row_prefix<<<gp, kThr, 0, s>>>(counts_dev, nx, ny, P);
    const size_t tsm = disk_tile_smem(pl.Hs, pl.Ws);
    if (tsm <= kDiskTileMaxSmem) {
        if ((e = cudaFuncSetAttribute(k_disk_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) !=
            cudaSuccess)
            return lc_cuda(e, "cudaFuncSetAttribute");
        const dim3 gt((unsigned)((nx + kDiskTX - 1) / kDiskTX),
                      (unsigned)std::min<int64_t>(((int64_t)ny + kDiskTY - 1) / kDiskTY, 65535));
        k_disk_tile<<<gt, kThr, tsm, s>>>(P, nx, ny, half, pl.Hs, pl.Ws, scale / (double)pl.count, out_dev);
    } else {
        const dim3 gd((unsigned)((nx + kThr - 1) / kThr), (unsigned)std::min<int64_t>(ny, 65535));
        k_disk<<<gd, kThr, (size_t)(2 * pl.Hs + 1) * sizeof(int), s>>>(P, nx, ny, half, pl.Hs,
                                                                        scale / (double)pl.count, out_dev);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return lc_cuda(e, "disk launches");
    return MLENS_OK;
}

}  // namespace
}  // namespace mlens

extern "C" {

int mlens_convolve_workspace(const mlens_grid *src, int32_t profile, double size, uint64_t *bytes_out)
{
    if (!bytes_out) return lc_fail(MLENS_ERR_ARG, "bytes_out is NULL");
    ConvPlan pl;
    int rc;
    if ((rc = plan_convolution(src, profile, size, &pl))) return rc;
    *bytes_out = pl.bytes;
    return MLENS_OK;
}

int mlens_convolve(const uint32_t *counts_dev, const mlens_grid *src, int32_t profile, double size, double scale,
                   float *out_dev, void *work_dev, uint64_t work_bytes, void *stream)
{
    ConvPlan pl;
    int rc;
    if ((rc = plan_convolution(src, profile, size, &pl))) return rc;
    if (!counts_dev || !out_dev) return lc_fail(MLENS_ERR_ARG, "counts_dev and out_dev must be non-NULL");
    if (((uintptr_t)counts_dev & 3u) || ((uintptr_t)out_dev & 3u))
        return lc_fail(MLENS_ERR_ARG, "counts_dev and out_dev must be 4-byte aligned");
    if (!std::isfinite(scale)) return lc_fail(MLENS_ERR_ARG, "scale must be finite");
    const int64_t npix = (int64_t)src->nx * src->ny;
    const uintptr_t a0 = (uintptr_t)counts_dev, a1 = a0 + 4 * (uintptr_t)npix;
    const uintptr_t b0 = (uintptr_t)out_dev, b1 = b0 + 4 * (uintptr_t)npix;
    if (a0 < b1 && b0 < a1) return lc_fail(MLENS_ERR_ARG, "out_dev must not overlap counts_dev");
    if (work_dev) {
        if (((uintptr_t)work_dev & 255u) != 0) return lc_fail(MLENS_ERR_ARG, "work_dev must be 256-byte aligned");
        if (work_bytes < pl.bytes) return lc_fail(MLENS_ERR_ARG, "work_bytes is below mlens_convolve_workspace's size");
        const uintptr_t w0 = (uintptr_t)work_dev, w1 = w0 + pl.bytes;
        if ((w0 < a1 && a0 < w1) || (w0 < b1 && b0 < w1))
            return lc_fail(MLENS_ERR_ARG, "work_dev must not overlap counts_dev or out_dev");
        return run_convolution(counts_dev, src, profile, size, scale, out_dev, pl, (char *)work_dev,
                               (cudaStream_t)stream);
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *work = nullptr;
    cudaError_t e = dmalloc(&work, pl.bytes);
    if (e != cudaSuccess) return lc_cuda(e, "cudaMalloc(convolution workspace)");
    rc = run_convolution(counts_dev, src, profile, size, scale, out_dev, pl, work, s);
    e = cudaStreamSynchronize(s);
    dfree(work);
    if (rc == MLENS_OK && e != cudaSuccess) rc = lc_cuda(e, "cudaStreamSynchronize");
    return rc;
}

int mlens_light_curve(const float *map_dev, const mlens_grid *src, double bx0, double by0, double bx1, double by1,
                      int32_t npts, float *out_dev, void *stream)
{
    int rc;
    if ((rc = check_map(src))) return rc;
    if (npts < 1) return lc_fail(MLENS_ERR_ARG, "npts must be >= 1");
    if (!map_dev || !out_dev) return lc_fail(MLENS_ERR_ARG, "map_dev and out_dev must be non-NULL");
    if (((uintptr_t)map_dev & 3u) || ((uintptr_t)out_dev & 3u))
        return lc_fail(MLENS_ERR_ARG, "map_dev and out_dev must be 4-byte aligned");
    if (!std::isfinite(bx0) || !std::isfinite(by0) || !std::isfinite(bx1) || !std::isfinite(by1))
        return lc_fail(MLENS_ERR_ARG, "track end points must be finite");
    Track T;
    T.x0 = src->x0;
    T.y0 = src->y0;
    T.dx = (src->x1 - src->x0) / src->nx;
    T.dy = (src->y1 - src->y0) / src->ny;
    T.bx0 = bx0;
    T.by0 = by0;
    T.bx1 = bx1;
    T.by1 = by1;
    T.nx = src->nx;
    T.ny = src->ny;
    T.n = npts;
    k_curve<<<(unsigned)((npts + kThr - 1) / kThr), kThr, 0, (cudaStream_t)stream>>>(map_dev, T, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lc_cuda(e, "light curve launch");
    return MLENS_OK;
}

int mlens_magnification_scale(const mlens_grid *rays, const mlens_grid *src, double *scale_out)
{
    if (!rays || !src || !scale_out) return lc_fail(MLENS_ERR_ARG, "rays, src and scale_out must be non-NULL");
    int rc;
    if ((rc = check_map(src))) return rc;
    if (!(rays->x1 > rays->x0) || !(rays->y1 > rays->y0) || rays->nx < 1 || rays->ny < 1 ||
        !std::isfinite(rays->x1 - rays->x0) || !std::isfinite(rays->y1 - rays->y0))
        return lc_fail(MLENS_ERR_ARG, "rays grid needs a finite box with x1 > x0, y1 > y0 and nx, ny >= 1");
    const double a_lens = (rays->x1 - rays->x0) * (rays->y1 - rays->y0);
    const double dx = (src->x1 - src->x0) / src->nx, dy = (src->y1 - src->y0) / src->ny;
    *scale_out = a_lens / ((double)rays->nx * (double)rays->ny * dx * dy);
    return MLENS_OK;
}

}  // extern "C"
