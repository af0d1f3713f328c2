// Device helpers shared by the dexgb kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dexgb.h"

namespace dex {

// ---------------------------------------------------------------- status --
__device__ __forceinline__ void raise_status(unsigned int* status, unsigned int bits)
{
    if (status) atomicOr(status, bits);
}

// ---------------------------------------------------------- exponentials --
// 2^x on the SFU (MUFU.EX2); flush-to-zero for results below FLT_MIN.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Taylor coefficients of 1 - 2^x = -sum_{k>=1} (x ln2)^k / k!, built from ln 2.
constexpr double kLn2 = 0.69314718055994530942;
constexpr double taylor_coef(int k)
{
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c *= kLn2 / (double)i;
    return -c;
}
constexpr float kG1 = (float)taylor_coef(1);
constexpr float kG2 = (float)taylor_coef(2);
constexpr float kG3 = (float)taylor_coef(3);
constexpr float kG4 = (float)taylor_coef(4);
constexpr float kG5 = (float)taylor_coef(5);
// Series used for tau < 0.1, i.e. x = -tau log2(e) > -0.1443: the first dropped
// term is tau^6/720, a relative error below 2e-8.  Above it 1 - 2^x >= 0.095 and
// the SFU's few-ulp error in 2^x costs < 3e-6 relative.
constexpr float kSeriesCut = -0.14426950f;
constexpr float kNegLog2e = -1.4426950408889634f;

// Transparent emitters (chi = 0, eta > 0) are stored as chi = eta * 2^-60 and
// S = 2^60, so that S (1 - e^{-chi len}) = eta len (1 - O(eta len 2^-60)) with no
// per-wavelength branch in the solvers.  Exact to float32 for eta <= 2^36.
constexpr float kEmitterScale = 1.152921504606846976e18f;     // 2^60
constexpr float kEmitterInvScale = 8.673617379884035e-19f;    // 2^-60
constexpr float kEmitterMaxEta = 68719476736.0f;              // 2^36

// Record entry (S, chi) of a voxel with emissivity e and opacity c (both >= 0).
__host__ __device__ __forceinline__ void encode_voxel(float e, float c, float& S, float& chi)
{
    if (c > 0.0f) {
        S = e / c;
        chi = c;
    } else if (e > 0.0f) {
        S = kEmitterScale;
        chi = e * kEmitterInvScale;
    } else {
        S = 0.0f;
        chi = 0.0f;
    }
}

// One voxel segment of length `len` for one wavelength: the piecewise-constant
// solution of Eq. RteIntegral composited front to back (probe outward):
//   I += T * S * (1 - e^{-chi len});  T *= e^{-chi len}
// nl2 = -len log2(e) is shared by the wavelengths of a record.
__device__ __forceinline__ void segment(float S, float chi, float nl2, float& I, float& T)
{
    const float x = chi * nl2;             // -tau log2(e)
    const float e = ex2_approx(x);         // e^{-tau}
    float p = fmaf(x, kG5, kG4);
    p = fmaf(x, p, kG3);
    p = fmaf(x, p, kG2);
    p = fmaf(x, p, kG1);
    const float g = (x > kSeriesCut) ? x * p : 1.0f - e;  // 1 - e^{-tau}
    I = fmaf(T, S * g, I);
    T *= e;
}

// Ray parameter of grid planes as an unevaluated sum hi + lo of two floats.
// A plane at offset P (a half-integer, exact) from the origin along an axis
// with direction component d is hit at t = P / d.  hi = P * ih is the rounded
// product with ih = fl(1/d); lo collects the product's rounding error (exact
// through an FMA) plus P times the residual 1/d - ih.  Path lengths are then
// differences (hi_b - hi_a) + (lo_b - lo_a), accurate relative to the length
// itself rather than to t, which matters far from the origin (t ~ 1e3 cells has
// an fp32 ulp of ~1e-4 cell).
struct AxisParam {
    float ih;  // fl(1/d), +inf for d == 0
    float il;  // 1/d - ih
};

__device__ __forceinline__ AxisParam axis_param(float d)
{
    AxisParam a;
    if (d != 0.0f) {
        a.ih = 1.0f / d;
        a.il = fmaf(-d, a.ih, 1.0f) * a.ih;
    } else {
        a.ih = __int_as_float(0x7f800000);
        a.il = 0.0f;
    }
    return a;
}

// lo part of the parameter of plane P whose rounded value is hi = P * a.ih
__device__ __forceinline__ float plane_lo(float P, const AxisParam& a, float hi)
{
    return fmaf(P, a.il, fmaf(P, a.ih, -hi));
}

// Loads of one wavelength-batch record (2W floats, 8W-byte aligned).
template <int W>
struct Record {
    float S[W];
    float chi[W];
};

template <int W>
__device__ __forceinline__ Record<W> load_record(const float* __restrict__ p)
{
    Record<W> r;
    if constexpr (W == 8) {
        const float4* q = reinterpret_cast<const float4*>(p);
        float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
        r.S[0] = a.x; r.S[1] = a.y; r.S[2] = a.z; r.S[3] = a.w;
        r.S[4] = b.x; r.S[5] = b.y; r.S[6] = b.z; r.S[7] = b.w;
        r.chi[0] = c.x; r.chi[1] = c.y; r.chi[2] = c.z; r.chi[3] = c.w;
        r.chi[4] = d.x; r.chi[5] = d.y; r.chi[6] = d.z; r.chi[7] = d.w;
    } else if constexpr (W == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
        float4 a = __ldg(q), b = __ldg(q + 1);
        r.S[0] = a.x; r.S[1] = a.y; r.S[2] = a.z; r.S[3] = a.w;
        r.chi[0] = b.x; r.chi[1] = b.y; r.chi[2] = b.z; r.chi[3] = b.w;
    } else if constexpr (W == 2) {
        float4 a = __ldg(reinterpret_cast<const float4*>(p));
        r.S[0] = a.x; r.S[1] = a.y; r.chi[0] = a.z; r.chi[1] = a.w;
    } else {
        float2 a = __ldg(reinterpret_cast<const float2*>(p));
        r.S[0] = a.x; r.chi[0] = a.y;
    }
    return r;
}

// Quadrature passed by value to the solve kernels.
struct Quadrature {
    int n_dir;
    float dx[DEX_MAX_DIRS];
    float dz[DEX_MAX_DIRS];
    float w[DEX_MAX_DIRS];
};

}  // namespace dex
