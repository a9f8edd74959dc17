// shoot_fp64.cu -- IEEE FP64 variant of the direct sum (Eq. 3), the source
// position (Eq. 2) and the FP64 binning rule, with every operation written as
// an explicitly rounded intrinsic in the order the equations state it, stars
// visited in input order.  Its beta and its maps therefore equal a plain IEEE
// FP64 evaluation of the same formulas bit for bit.  On GB300 FP64 runs at a
// small fraction of the FP32 rate; this path exists for verification
// (mlens_trace), for the precision study and for exact per-ray references, not
// for throughput.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlens_dev.cuh"

namespace mlens {

constexpr int kT64 = 128;

__device__ __forceinline__ void alpha_fp64(double tx, double ty, const float4 *sq, int cnt, double &sx, double &sy)
{
    for (int k = 0; k < cnt; ++k) {
        const float4 q = sq[k];
        const double dx = __dsub_rn(tx, (double)q.x);
        const double dy = __dsub_rn(ty, (double)q.y);
        const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double m = (double)q.z;
        sx = __dadd_rn(sx, __ddiv_rn(__dmul_rn(m, dx), r2));
        sy = __dadd_rn(sy, __ddiv_rn(__dmul_rn(m, dy), r2));
    }
}

__device__ __forceinline__ double ray_coord(double x0, double x1, int n, int i)
{
    return __dadd_rn(x0, __dmul_rn(__dadd_rn((double)i, 0.5), __ddiv_rn(__dsub_rn(x1, x0), (double)n)));
}

__device__ __forceinline__ int pixel_fp64(double bx, double by, const BinGrid &g)
{
    if (!isfinite(bx) || !isfinite(by)) return -2;
    const double ux = floor(__dmul_rn(__dsub_rn(bx, g.x0), __ddiv_rn((double)g.nx, __dsub_rn(g.x1, g.x0))));
    const double uy = floor(__dmul_rn(__dsub_rn(by, g.y0), __ddiv_rn((double)g.ny, __dsub_rn(g.y1, g.y0))));
    if (ux < 0.0 || ux >= (double)g.nx || uy < 0.0 || uy >= (double)g.ny) return -1;
    return (int)uy * g.nx + (int)ux;
}

// GRID: rays of a grid (one per thread, 32 x 4 threads per CTA), binned;
// otherwise: k arbitrary positions from `theta`, beta written, nothing binned.
template <bool GRID>
__global__ void __launch_bounds__(kT64) k_fp64(ShootArgs a, const double2 *theta, double2 *beta, int64_t k, int by0)
{
    __shared__ float4 sq[kT64];
    __shared__ unsigned sred[3];
    const int tid = threadIdx.x;
    if (tid == 0) sred[0] = sred[1] = sred[2] = 0u;

    int i = 0, j = 0;
    int64_t r = 0;
    bool ok;
    double tx, ty;
    if (GRID) {
        i = blockIdx.x * 32 + (tid & 31);
        j = (by0 + (int)blockIdx.y) * 4 + (tid >> 5);
        ok = i < a.rays.nx && j < a.rays.ny;
        tx = ray_coord(a.rays.x0, a.rays.x1, a.rays.nx, i);
        ty = ray_coord(a.rays.y0, a.rays.y1, a.rays.ny, j);
    } else {
        r = (int64_t)blockIdx.x * kT64 + tid;
        ok = r < k;
        const double2 t = ok ? theta[r] : make_double2(0.0, 0.0);
        tx = t.x;
        ty = t.y;
    }
    const double kc = a.lens.kc, g1 = a.lens.g1, g2 = a.lens.g2;
    double sx = __dadd_rn(__dmul_rn(__dadd_rn(kc, g1), tx), __dmul_rn(g2, ty));
    double sy = __dadd_rn(__dmul_rn(g2, tx), __dmul_rn(__dsub_rn(kc, g1), ty));
    for (int64_t s0 = 0; s0 < a.nstars; s0 += kT64) {
        const int cnt = (int)min((int64_t)kT64, a.nstars - s0);
        __syncthreads();
        if (tid < cnt) sq[tid] = a.stars[s0 + tid];
        __syncthreads();
        alpha_fp64(tx, ty, sq, cnt, sx, sy);
    }
    const double bx = __dsub_rn(tx, sx), by = __dsub_rn(ty, sy);
    if (!GRID) {
        if (ok) beta[r] = make_double2(bx, by);
        return;
    }
    unsigned nb = 0, no = 0, nn = 0;
    if (ok) {
        const int p = pixel_fp64(bx, by, a.bin);
        if (p >= 0) {
            atomicAdd(&a.counts[p], 1u);
            nb = 1;
        } else if (p == -1) {
            no = 1;
        } else {
            nn = 1;
        }
        if (a.beta_out) reinterpret_cast<double2 *>(a.beta_out)[(int64_t)j * a.rays.nx + i] = make_double2(bx, by);
    }
    __syncthreads();
    stats_add_block(nb, no, nn, sred, a.stats);
}

cudaError_t launch_shoot_fp64(const ShootArgs &a, cudaStream_t s, int row0, int row1)
{
    // blocks of 32 x 4 rays: rows [row0, row1) in block rows (row0 a multiple of 4)
    const int tx = (a.rays.nx + 31) / 32;
    const int r1 = row1 < 0 || row1 > a.rays.ny ? a.rays.ny : row1;
    const int ty = (r1 + 3) / 4;
    for (int by0 = row0 / 4; by0 < ty; by0 += 65535) {
        const dim3 grid((unsigned)tx, (unsigned)min(65535, ty - by0));
        k_fp64<true><<<grid, kT64, 0, s>>>(a, nullptr, nullptr, 0, by0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_trace_fp64(const float4 *stars, int64_t nstars, const LensTerms &lens, const double2 *theta,
                              double2 *beta, int64_t k, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    ShootArgs a{};
    a.stars = stars;
    a.nstars = nstars;
    a.lens = lens;
    int64_t nb = (k + kT64 - 1) / kT64;
    if (nb > 0x7fffffff) return cudaErrorInvalidConfiguration;
    k_fp64<false><<<(unsigned)nb, kT64, 0, s>>>(a, theta, beta, k, 0);
    return cudaGetLastError();
}

}  // namespace mlens
