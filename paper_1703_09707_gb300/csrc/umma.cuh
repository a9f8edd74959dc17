// umma.cuh -- Blackwell fifth-generation tensor-core helpers (tcgen05, inline
// PTX): tensor-memory allocation, shared-memory matrix descriptors for K-major
// and MN-major operands without swizzle, the BF16 -> FP32 MMA, its commit to an mbarrier,
// a bounded wait, and accumulator loads.
//
// Operand layout ("core matrices"): a K-major [R][64] BF16 operand is stored as
// 8-row x 16-byte core matrices; core matrix (r / 8, k / 8) starts at
// (r / 8) * 1024 + (k / 8) * 128 bytes and row r % 8 of it at + 16 (r % 8).
// In descriptor terms the leading-dimension (K) offset is 128 bytes and the
// stride-dimension (M/N) offset 1024 bytes; one MMA consumes K = 16, i.e. the
// next two core matrices along K (+256 bytes per step).
//
// An MN-major operand (instruction-descriptor transpose bit) has core matrices of
// 8 K-rows x 16 bytes along M/N.  Without swizzle its descriptor takes the same
// roles as a K-major one: the leading-dimension offset is the stride between core
// matrices along K and the stride-dimension offset the stride along M/N (measured
// on GB300 with an M = 128, N = 64, K = 16 product against a host reference: the
// other assignment gives a different product).  So a row-major block of 8 x 8
// core matrices [rows][cols] serves both as a K-major operand over its columns
// and as an MN-major operand over its rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mlens {
namespace umma {

__host__ __device__ constexpr int cm_offset(int r, int k)
{
    return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, version 1).
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, shape
// M x N; A and B K-major unless a_mn / b_mn (MN-major).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, bool a_mn = false, bool b_mn = false)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Whole warp: allocate ncols tensor-memory columns, address written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One thread: D (tensor memory) = A B^T, or += when accumulate != 0.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One thread: arrive on *bar once the MMAs it issued have completed.
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Wait for phase `parity` of *bar, giving up after max_iter polls; true if it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int max_iter)
{
    uint32_t done = 0;
    for (int it = 0; it < max_iter && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
    return done != 0;
}

// Whole warp: 16 consecutive FP32 accumulator columns of this warp's 32 lanes
// (warp w of a warpgroup reads lanes 32 (w % 4) .. + 31; taddr carries the lane
// base in bits 31..16).
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Named barrier over the 128 threads of warpgroup wg (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void wg_sync(int wg)
{
    if (wg == 0)
        asm volatile("bar.sync 1, 128;" ::: "memory");
    else
        asm volatile("bar.sync 2, 128;" ::: "memory");
}

}  // namespace umma
}  // namespace mlens
