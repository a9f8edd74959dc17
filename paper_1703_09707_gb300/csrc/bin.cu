// bin.cu -- the binning step of Algorithm 1 on its own: float-pair source
// positions -> exact pixel -> warp-aggregated, shared-memory-privatised
// window histogram -> global uint32 counts.  Same rule and same epilogue as
// the fused shooting kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_dev.cuh"

namespace mlens {

constexpr int kBinThreads = 256;
constexpr int kBinPer = 8;  // records per thread; a CTA takes 2048 consecutive records

__global__ void __launch_bounds__(kBinThreads) k_bin(BinArgs a)
{
    __shared__ uint32_t hist[kWin * kWin];
    __shared__ int win[2];
    __shared__ unsigned sred[3];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kBinThreads * kBinPer;
    for (int b = tid; b < kWin * kWin; b += kBinThreads) hist[b] = 0u;
    if (tid == 0) {
        sred[0] = sred[1] = sred[2] = 0u;
        // window on the first finite record of this CTA's range (rays of one grid
        // row segment land close together)
        int wx = -(1 << 30), wy = -(1 << 30);
        for (int r = 0; r < kBinThreads * kBinPer && base + r < a.n; ++r) {
            float4 v = a.beta[base + r];
            if (isfinite(v.x) && isfinite(v.y)) {
                wx = pair_axis_rough(v.x, a.bin.ax) - kWin / 2;
                wy = pair_axis_rough(v.y, a.bin.ay) - kWin / 2;
                break;
            }
        }
        win[0] = wx;
        win[1] = wy;
    }
    __syncthreads();
    WinHist W{hist, win[0], win[1]};
    unsigned nb = 0, no = 0, nn = 0;
#pragma unroll
    for (int r = 0; r < kBinPer; ++r) {
        const int64_t idx = base + (int64_t)r * kBinThreads + tid;  // coalesced
        uint32_t key = kNoKey;
        if (idx < a.n) {
            const float4 v = a.beta[idx];
            int gpx = 0, gpy = 0;
            const int pix = pair_pixel(v.x, v.y, v.z, v.w, a.bin, gpx, gpy);
            if (pix >= 0) {
                ++nb;
                key = hist_key(pix, gpx, gpy, W, a.bin);
            } else if (pix == -1) {
                ++no;
            } else {
                ++nn;
            }
        }
        hist_add_warp(key, W, a.counts);
    }
    __syncthreads();
    hist_flush(W, a.bin, a.counts);
    stats_add_block(nb, no, nn, sred, a.stats);
}

cudaError_t launch_bin(const BinArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const int64_t per = (int64_t)kBinThreads * kBinPer;
    const int64_t nb = (a.n + per - 1) / per;
    if (nb > 0x7fffffff) return cudaErrorInvalidConfiguration;
    k_bin<<<(unsigned)nb, kBinThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mlens
