// mlp.cuh -- the far-field network of the learned-far-field variant: sizes,
// parameter layout and activations.  Its products run on the fifth-generation
// tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation; umma.cuh).
//
// Network: a per-cell latent z (32) and one shared MLP 34 -> 64 -> 64 -> 2,
//   h1 = W1z z + W1u u + b1, a1 = silu(h1); h2 = W2 a1 + b2, a2 = silu(h2);
//   y = W3 a2 + b3,  silu(v) = v (1 + tanh(v/2)) / 2 (tanh from the hardware unit).
// The latent block of layer 1 and layer 2 run on the tensor cores with BF16
// operands (z, W1z, a1, W2; dh2, dh1 in the backward pass); the position block
// of layer 1 (W1u u, 2 inputs) and layer 3 stay in FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mlens {
namespace mlp {

constexpr int kLat = 32;
constexpr int kHid = 64;
constexpr int kOut = 2;
// flat FP32 parameter layout
constexpr int oW1z = 0;                      // [64][32]
constexpr int oW1u = oW1z + kHid * kLat;     // [64][2]
constexpr int ob1 = oW1u + kHid * 2;         // [64]
constexpr int oW2 = ob1 + kHid;              // [64][64]
constexpr int ob2 = oW2 + kHid * kHid;       // [64]
constexpr int oW3 = ob2 + kHid;              // [2][64]
constexpr int ob3 = oW3 + kOut * kHid;       // [2]
constexpr int kParams = ob3 + kOut;          // 6530

// sigma(v) = (1 + tanh(v/2)) / 2 from the hardware tanh (MUFU.TANH, one
// special-function op; maximum relative error about 2^-11, below the 2^-8
// resolution of the BF16 operands the activations feed).  The accurate tanhf
// costs about 20 instructions and, at 128 activations per ray, dominated the
// learned kernel.  Training and inference use the same function.
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// layer 2 may keep the accurate tanhf (its outputs feed the FP32 layer 3)
constexpr bool kLayer2Hw = true;
__device__ __forceinline__ float sigm_hw(float v) { return __fmaf_rn(0.5f, tanh_hw(0.5f * v), 0.5f); }
__device__ __forceinline__ float sigm_acc(float v) { return 0.5f * (1.0f + tanhf(0.5f * v)); }
__device__ __forceinline__ float sigm2(float v) { return kLayer2Hw ? sigm_hw(v) : sigm_acc(v); }
// v sigma(v) = h + h tanh(h) with h = v / 2: three instructions with the hardware tanh
__device__ __forceinline__ float silu_hw(float v)
{
    const float h = 0.5f * v;
    return __fmaf_rn(h, tanh_hw(h), h);
}
__device__ __forceinline__ float silu1(float v) { return silu_hw(v); }
__device__ __forceinline__ float silu2(float v) { return kLayer2Hw ? silu_hw(v) : v * sigm_acc(v); }
__device__ __forceinline__ float dsilu1(float v)
{
    const float s = sigm_hw(v);
    return s * (1.0f + v * (1.0f - s));
}
__device__ __forceinline__ float dsilu2(float v)
{
    const float s = sigm2(v);
    return s * (1.0f + v * (1.0f - s));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&p);
}

__device__ __forceinline__ __nv_bfloat16 to_bf16(float v) { return __float2bfloat16_rn(v); }

}  // namespace mlp
}  // namespace mlens
