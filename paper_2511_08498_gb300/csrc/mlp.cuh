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

// GELU, tanh form: g(z) = z/2 (1 + tanh(c (z + k z^3))), c = sqrt(2/pi), k = 0.044715
__device__ __forceinline__ Act gelu(float z)
{
    const float c = 0.79788456080286536f, k = 0.044715f;
    const float z2 = z * z;
    const float t = tanhf(c * fmaf(k * z2, z, z));
    Act r;
    r.g = 0.5f * z * (1.0f + t);
    r.dg = fmaf(0.5f * z * (1.0f - t * t) * c, fmaf(3.0f * k, z2, 1.0f), 0.5f * (1.0f + t));
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
