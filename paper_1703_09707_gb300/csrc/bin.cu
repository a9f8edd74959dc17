// bin.cu -- the binning step of Algorithm 1 on its own: float-pair source
// positions -> exact pixel -> shared-memory-privatised window histogram -> global
// uint32 counts.  Same pixel rule and window as the fused shooting kernels; one
// atomic per record instead of their warp run aggregation (here, without a star
// sum to hide it, the aggregation's shuffle, vote and branch per record cost more
// than the atomics it saves: 0.336 -> 0.303 ms grid order, 0.309 -> 0.281 ms flat
// order for 8192^2 records).
//
// Two record orders.  Flat: a CTA takes 4096 consecutive records.  Grid: the
// records are a row-major nx x ny ray grid and a CTA takes a 64 x 64 block of
// it; neighbouring rays land on neighbouring pixels, so most of the block's
// records hit its 64 x 64 window, placed on the record nearest the block's
// centre (consecutive records of one grid row would instead spread along a
// strip of the map far longer than the window).
//
// The kernel is issue-bound (~100 instructions per 16-byte record), not
// bandwidth-bound: staging the records through shared memory by bulk copies,
// prefetching them into L2, or larger blocks per CTA all measured slower than
// loading each thread's records straight to registers, 8 in flight at a time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_dev.cuh"

namespace mlens {

constexpr int kBinThreads = 256;
constexpr int kBinPer = 8;                                    // records per thread and round
constexpr int kBinRounds = 2;                                 // the window is placed after round 0's loads
constexpr int kBinRecs = kBinThreads * kBinPer * kBinRounds;  // 4096 records per CTA
constexpr int kBinTileX = 64;                                 // grid order: 64 x 64 records per CTA
constexpr int kBinTileY = kBinRecs / kBinTileX;
constexpr int kBinRowStep = kBinThreads / kBinTileX;          // rows between a thread's records

// Record r (0 <= r < kBinPer * kBinRounds) of thread tid: index, validity, and a
// placement priority (unique per record; lowest = nearest the block's centre in
// grid order, first in flat order).
template <bool GRID>
__device__ __forceinline__ int64_t bin_record(const BinArgs &a, int tid, int r, bool &ok, unsigned &prio)
{
    if (GRID) {
        const int c = tid % kBinTileX, rr = tid / kBinTileX + r * kBinRowStep;
        const int col = blockIdx.x * kBinTileX + c;
        const int64_t row = (int64_t)blockIdx.y * kBinTileY + rr;
        ok = col < a.rnx && row < a.rny;
        prio = ((unsigned)(abs(rr - kBinTileY / 2) + abs(c - kBinTileX / 2)) << 12) | (unsigned)(rr * kBinTileX + c);
        return row * a.rnx + col;  // a warp reads 32 consecutive records of one row
    }
    const int64_t idx = (int64_t)blockIdx.x * kBinRecs + (int64_t)r * kBinThreads + tid;
    ok = idx < a.n;
    prio = (unsigned)(r * kBinThreads + tid);
    return idx;
}

// The exact rule for a record whose quick tests were inconclusive (a few per
// million, and every record with a non-finite component), out of line so that
// the unrolled record loop stays small.
struct BinPix {
    int pix, px, py;  // pix: linear pixel, -1 outside the map, -2 non-finite
};

__device__ __noinline__ BinPix bin_pixel_exact(float xh, float yh, float xl, float yl, AxisPair ax, AxisPair ay)
{
    BinPix p{-2, -1, -1};
    if (!isfinite(xh) || !isfinite(yh) || !isfinite(xl) || !isfinite(yl)) return p;
    p.px = pair_axis_exact(xh, xl, ax);
    p.py = pair_axis_exact(yh, yl, ay);
    p.pix = (p.px < 0 || p.py < 0) ? -1 : p.py * ax.n + p.px;
    return p;
}

// Classify one record (ok = it exists) and add it to the histogram.  Both quick
// tests pass only when all four components are finite, so the common path needs
// no finiteness test.
template <bool GRID>
__device__ __forceinline__ void bin_one(const BinArgs &a, const float4 &v, bool ok, const WinHist &W, unsigned &nb,
                                        unsigned &no, unsigned &nn)
{
    int px, py, pix;
    const bool qx = pair_axis_quick(v.x, v.z, a.bin.ax, px);
    const bool qy = pair_axis_quick(v.y, v.w, a.bin.ay, py);
    if (qx && qy) {
        pix = (px | py) < 0 ? -1 : py * a.bin.nx + px;
    } else {
        const BinPix p = bin_pixel_exact(v.x, v.y, v.z, v.w, a.bin.ax, a.bin.ay);
        pix = p.pix;
        px = p.px;
        py = p.py;
    }
    if (!ok) pix = -3;
    nb += pix >= 0;
    no += pix == -1;
    nn += pix == -2;
    uint32_t key = kNoKey;
    if (pix >= 0) {
        const unsigned wx = (unsigned)(px - W.wx0), wy = (unsigned)(py - W.wy0);
        key = (wx < (unsigned)kWin && wy < (unsigned)kWin) ? wy * kWin + wx : (uint32_t)(kWin * kWin) + (uint32_t)pix;
    }
    if (key != kNoKey) {  // one atomic per record
        if (key < (uint32_t)(kWin * kWin))
            atomicAdd(&W.h[key], 1u);
        else
            atomicAdd(&a.counts[key - (uint32_t)(kWin * kWin)], 1u);
    }
}

template <bool GRID>
__device__ __forceinline__ void bin_block(const BinArgs &a)
{
    __shared__ __align__(16) uint32_t hist[kWin * kWin];
    __shared__ int win[2];
    __shared__ unsigned wq;
    __shared__ unsigned sred[3];
    const int tid = threadIdx.x;
    hist_zero(hist);
    if (tid == 0) {
        wq = 0xffffffffu;
        sred[0] = sred[1] = sred[2] = 0u;
    }
    __syncthreads();

    // round 0: loads first (all in flight together), then the window
    float4 v[kBinPer];
    bool ok[kBinPer];
    unsigned best = 0xffffffffu;
#pragma unroll
    for (int r = 0; r < kBinPer; ++r) {
        unsigned prio;
        const int64_t idx = bin_record<GRID>(a, tid, r, ok[r], prio);
        v[r] = ok[r] ? a.beta[idx] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int r = 0; r < kBinPer; ++r) {
        bool okr;
        unsigned prio;
        bin_record<GRID>(a, tid, r, okr, prio);
        if (ok[r] && isfinite(v[r].x) && isfinite(v[r].y)) best = min(best, prio);
    }
    const unsigned wbest = __reduce_min_sync(0xffffffffu, best);
    if ((tid & 31) == 0 && wbest != 0xffffffffu) atomicMin(&wq, wbest);
    __syncthreads();
    const unsigned q = wq;
    if (q == 0xffffffffu) {
        if (tid == 0) win[0] = win[1] = -(1 << 30);  // no finite record: every key is global
    } else {
#pragma unroll
        for (int r = 0; r < kBinPer; ++r) {
            bool okr;
            unsigned prio;
            bin_record<GRID>(a, tid, r, okr, prio);
            if (prio == q) {
                win[0] = pair_axis_rough(v[r].x, a.bin.ax) - kWin / 2;
                win[1] = pair_axis_rough(v[r].y, a.bin.ay) - kWin / 2;
            }
        }
    }
    __syncthreads();
    const WinHist W{hist, win[0], win[1]};
    unsigned nb = 0, no = 0, nn = 0;
#pragma unroll
    for (int r = 0; r < kBinPer; ++r) bin_one<GRID>(a, v[r], ok[r], W, nb, no, nn);

#pragma unroll
    for (int k = 1; k < kBinRounds; ++k) {
#pragma unroll
        for (int r = 0; r < kBinPer; ++r) {
            unsigned prio;
            const int64_t idx = bin_record<GRID>(a, tid, k * kBinPer + r, ok[r], prio);
            v[r] = ok[r] ? a.beta[idx] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int r = 0; r < kBinPer; ++r) bin_one<GRID>(a, v[r], ok[r], W, nb, no, nn);
    }
    __syncthreads();
    hist_flush(W, a.bin, a.counts);
    stats_add_block(nb, no, nn, sred, a.stats);
}

// Resident CTAs per SM: four in both orders (flat order at five CTAs, 48 registers,
// spilled and ran 2 % slower; grid order keeps the 64 registers it takes).
__global__ void __launch_bounds__(kBinThreads) k_bin_grid(BinArgs a) { bin_block<true>(a); }
__global__ void __launch_bounds__(kBinThreads, 4) k_bin_flat(BinArgs a) { bin_block<false>(a); }

cudaError_t launch_bin(const BinArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    if (a.rnx > 0) {
        const int64_t tx = (a.rnx + kBinTileX - 1) / kBinTileX, ty = (a.rny + kBinTileY - 1) / kBinTileY;
        if (tx > 0x7fffffff || ty > 65535) return cudaErrorInvalidConfiguration;
        k_bin_grid<<<dim3((unsigned)tx, (unsigned)ty), kBinThreads, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int64_t nb = (a.n + kBinRecs - 1) / kBinRecs;
    if (nb > 0x7fffffff) return cudaErrorInvalidConfiguration;
    k_bin_flat<<<(unsigned)nb, kBinThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mlens
