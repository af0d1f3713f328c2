// The profile-surrogate network shared by its tensor-core kernels (k_mlp.cu)
// and by the Core-and-Voigt solve that evaluates it per segment (k_cav.cu).
//   features f = (x / 16, log10(a) + 2, u / 16)
//   h1 = GELU(W1 f + b1) (64), h2 = GELU(W2 h1 + b2) (64), y = w3 . h2 + b3 ~ ln H(a, x - u)
// Parameter layout (floats): W1 [64][3] at 0, b1 at 192, W2 [64][64] (row = output)
// at 256, b2 at 4352, w3 at 4416, b3 at 4480.
#pragma once

#include <cuda_runtime.h>

namespace dex {
namespace mlp {

constexpr int kH = 64;
constexpr int kW1 = 0, kB1 = 192, kW2 = 256, kB2 = 4352, kW3 = 4416, kB3 = 4480, kParams = 4481;

// training domain of the surrogate (outside it the exact evaluation is used)
constexpr float kXMax = 16.0f, kUMax = 10.0f, kAMin = 1e-3f, kAMax = 1e-1f;

struct Act {
    float g, dg;
};

// GELU, tanh form: g(z) = z/2 (1 + tanh(u)), u = c (z + k z^3), c = sqrt(2/pi),
// k = 0.044715.  Evaluated through the identity 1/2 (1 + tanh u) = 1 / (1 + e^{-2u})
// (the logistic function of 2u): s = 1 / (1 + 2^{-2u log2 e}) with the
// special-function unit's 2^x and reciprocal, g = z s.  Nothing cancels, so s and
// g carry a few float32 ulps of relative error for every z (a large -2u makes
// 2^x overflow to +inf and s = 0, g = 0; a large u makes 2^x flush to 0 and s = 1).
//   g' = s + z s (1 - s) 2 u',  u' = c (1 + 3 k z^2).
__device__ __forceinline__ float mlp_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mlp_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ Act gelu(float z)
{
    const float c = 0.79788456080286536f, k = 0.044715f;
    const float m2log2e = -2.8853900817779268f;  // -2 log2(e)
    const float z2 = z * z;
    const float u = c * z * fmaf(k, z2, 1.0f);
    const float s = mlp_rcp(1.0f + mlp_ex2(u * m2log2e));
    Act r;
    r.g = z * s;
    r.dg = fmaf(z * s * (1.0f - s), 2.0f * c * fmaf(3.0f * k, z2, 1.0f), s);
    return r;
}

__device__ __forceinline__ void features(float x, float a, float u, float* f)
{
    f[0] = x * 0.0625f;
    f[1] = log10f(a) + 2.0f;
    f[2] = u * 0.0625f;
}

// Whole network in float32 on the CUDA cores (one sample per thread); w holds
// the parameters with W1, W2, w3 already rounded to bfloat16 values.
__device__ __forceinline__ float ln_h_fp32(const float* __restrict__ w, float x, float a, float u)
{
    float f[3];
    features(x, a, u, f);
    float h1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i)
        h1[i] = gelu(fmaf(w[kW1 + 3 * i + 2], f[2], fmaf(w[kW1 + 3 * i + 1], f[1], fmaf(w[kW1 + 3 * i], f[0], w[kB1 + i]))))
                    .g;
    float y = w[kB3];
#pragma unroll 1
    for (int j = 0; j < kH; ++j) {
        const float* row = w + kW2 + kH * j;
        float z = w[kB2 + j];
#pragma unroll
        for (int i = 0; i < kH; ++i) z = fmaf(row[i], h1[i], z);
        y = fmaf(w[kW3 + j], gelu(z).g, y);
    }
    return y;
}

}  // namespace mlp
}  // namespace dex
