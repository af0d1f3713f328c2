// Device helpers shared by the dexgb kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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
// 1 - e^{-tau} without a branch: g = min(P5(tau), (1 + 2^-21) - e), where
//  * P5 = tau - tau^2/2 + tau^3/6 - tau^4/24 + tau^5/120 (the series above in
//    x = -tau log2(e)) is never below 1 - e^{-tau} for tau >= 0 (the Lagrange
//    remainder -e^{-xi} tau^6/720 is negative) and exceeds it by tau^6/720;
//  * (1 + 2^-21) - e, with e = 2^x from the SFU (a few float ulps of error near
//    1, each ulp 2^-24 there), exceeds it by 2^-21 minus that error: an upper
//    bound while the error is below 2^-21 (8 such ulps), and within 2^-20 of it.
// The smaller of the two: the series wherever it is within ~5e-7 of the exact
// value (tau below ~0.27; relative error < 3e-7 for tau < 0.1), else 1 - e
// plus at most 2^-20.  Worst relative error, at the crossover near tau = 0.27:
// 2.2e-6 with an exact 2^x, 3.8e-6 with 2^x off by 2^-21 (the float32 model of
// this is tests/test_update_bound.py); < 5e-7 once g ~ 1.
// Compared with a select on tau, the min saves a compare and a select per
// wavelength; on the issue-bound 1024^2 benchmark solve it measured -3.4%.
constexpr float kOnePlus2m21 = 1.000000476837158203125f;  // 1 + 2^-21
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
    const float g = fminf(x * p, kOnePlus2m21 - e);  // 1 - e^{-tau}
    I = fmaf(T, S * g, I);
    T *= e;
}

// The same update for two wavelengths at once on the packed FP32 pipe
// (FFMA2/FMUL2/FADD2 of sm_100+): every lane of a pair is rounded exactly as
// in segment(), so results are bit-identical, with about half the FP32
// instructions issued.
__device__ __forceinline__ void segment2(float2 S, float2 chi, float nl2, float& I0, float& I1, float& T0,
                                         float& T1)
{
    const float2 x = __fmul2_rn(chi, make_float2(nl2, nl2));
    const float2 e = make_float2(ex2_approx(x.x), ex2_approx(x.y));
    float2 p = __ffma2_rn(x, make_float2(kG5, kG5), make_float2(kG4, kG4));
    p = __ffma2_rn(x, p, make_float2(kG3, kG3));
    p = __ffma2_rn(x, p, make_float2(kG2, kG2));
    p = __ffma2_rn(x, p, make_float2(kG1, kG1));
    const float2 xp = __fmul2_rn(x, p);
    const float2 ome = __fadd2_rn(make_float2(kOnePlus2m21, kOnePlus2m21), make_float2(-e.x, -e.y));
    const float2 g = make_float2(fminf(xp.x, ome.x), fminf(xp.y, ome.y));
    const float2 I = __ffma2_rn(make_float2(T0, T1), __fmul2_rn(S, g), make_float2(I0, I1));
    const float2 T = __fmul2_rn(make_float2(T0, T1), e);
    I0 = I.x;
    I1 = I.y;
    T0 = T.x;
    T1 = T.y;
}

// True when every transmission is exactly zero (underflowed): from then on each
// update adds T S (1 - e) = 0 and keeps T = 0, so the rest of the ray changes nothing.
template <int W>
__device__ __forceinline__ bool all_opaque(const float* T)
{
    unsigned int bits = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) bits |= __float_as_uint(T[w]);
    return bits == 0u;
}

// All W wavelengths of a record: pairs on the packed pipe, an odd one alone.
template <int W>
__device__ __forceinline__ void segments(const float* S, const float* chi, float nl2, float* I, float* T)
{
#pragma unroll
    for (int w = 0; w + 1 < W; w += 2)
        segment2(make_float2(S[w], S[w + 1]), make_float2(chi[w], chi[w + 1]), nl2, I[w], I[w + 1], T[w], T[w + 1]);
    if constexpr (W % 2 == 1) segment(S[W - 1], chi[W - 1], nl2, I[W - 1], T[W - 1]);
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

// 256-bit global loads (sm_100 and later): one 32-byte access per lane, so a
// warp reading 32 neighbouring 64-byte records touches each 32-byte sector once
// (four 128-bit loads touch every sector twice).  p must be 32-byte aligned.
__device__ __forceinline__ void ldg256(const float* __restrict__ p, float* v)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

__device__ __forceinline__ void ldg256u(const void* __restrict__ p, unsigned int* v)
{
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "l"(p));
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

// Storage formats of a static record (FP32 accumulation along the ray in all):
//   F32  : S[W], chi[W] float32 (8W bytes)
//   BF16 : S[W], chi[W] bfloat16, round to nearest even (4W bytes; W = 4, 8)
//   F16  : float32 scales (max S, max chi of the record), 2 pad words, then
//          S[W] / scaleS and chi[W] / scalechi as float16 (16 + 4W bytes; W = 4, 8)
enum StorageFormat { kStoreF32 = 0, kStoreBF16 = 1, kStoreF16 = 2 };

template <int W, int ST>
struct RecFmt;

template <int W>
struct RecFmt<W, kStoreF32> {
    static constexpr int kStride = 2 * W;  // floats
    // W = 8 and kWide: two 256-bit loads (the record must be 32-byte aligned);
    // otherwise load_record (128-bit loads)
    template <bool kWide = true>
    __device__ __forceinline__ static Record<W> load(const float* p)
    {
        if constexpr (W == 8 && kWide) {
            Record<W> r;
            ldg256(p, r.S);
            ldg256(p + 8, r.chi);
            return r;
        } else {
            return load_record<W>(p);
        }
    }
    __device__ __forceinline__ static void store(float* rec, const float* S, const float* chi)
    {
        if constexpr (W >= 2) {
            float4* q = reinterpret_cast<float4*>(rec);
            float v[2 * W];
#pragma unroll
            for (int w = 0; w < W; ++w) { v[w] = S[w]; v[W + w] = chi[w]; }
#pragma unroll
            for (int u = 0; u < (2 * W) / 4; ++u) q[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        } else {
            *reinterpret_cast<float2*>(rec) = make_float2(S[0], chi[0]);
        }
    }
};

template <int W>
struct RecFmt<W, kStoreBF16> {
    static_assert(W == 4 || W == 8, "reduced-precision records need W = 4 or 8");
    static constexpr int kStride = W;  // floats (2W bfloat16)
    __device__ __forceinline__ static float lo(unsigned int u) { return __uint_as_float(u << 16); }
    __device__ __forceinline__ static float hi(unsigned int u) { return __uint_as_float(u & 0xffff0000u); }
    template <bool kWide = true>
    __device__ __forceinline__ static Record<W> load(const float* p)
    {
        Record<W> r;
        const uint4* q = reinterpret_cast<const uint4*>(p);
        unsigned int u[W];
        if constexpr (W == 8 && kWide) {
            ldg256u(p, u);  // one 256-bit load (the record must be 32-byte aligned)
        } else if constexpr (W == 8) {
            const uint4 a = __ldg(q), b = __ldg(q + 1);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w; u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
        } else {
            const uint4 a = __ldg(q);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
        }
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            r.S[2 * k] = lo(u[k]);
            r.S[2 * k + 1] = hi(u[k]);
            r.chi[2 * k] = lo(u[W / 2 + k]);
            r.chi[2 * k + 1] = hi(u[W / 2 + k]);
        }
        return r;
    }
    __device__ __forceinline__ static void store(float* rec, const float* S, const float* chi)
    {
        unsigned int u[W];
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            u[k] = (unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(S[2 * k])) |
                   ((unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(S[2 * k + 1])) << 16);
            u[W / 2 + k] = (unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(chi[2 * k])) |
                           ((unsigned int)__bfloat16_as_ushort(__float2bfloat16_rn(chi[2 * k + 1])) << 16);
        }
        uint4* q = reinterpret_cast<uint4*>(rec);
#pragma unroll
        for (int k = 0; k < W / 4; ++k) q[k] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
    }
};

template <int W>
struct RecFmt<W, kStoreF16> {
    static_assert(W == 4 || W == 8, "reduced-precision records need W = 4 or 8");
    static constexpr int kStride = 4 + W;  // floats: 2 scales, 2 pad, 2W float16
    __device__ __forceinline__ static float h(unsigned int u, int hi_half)
    {
        return __half2float(__ushort_as_half((unsigned short)(hi_half ? (u >> 16) : (u & 0xffffu))));
    }
    template <bool kWide = true>  // 48-byte records: 128-bit loads only
    __device__ __forceinline__ static Record<W> load(const float* p)
    {
        Record<W> r;
        const float4 hd = __ldg(reinterpret_cast<const float4*>(p));
        const uint4* q = reinterpret_cast<const uint4*>(p + 4);
        unsigned int u[W];
        if constexpr (W == 8) {
            const uint4 a = __ldg(q), b = __ldg(q + 1);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w; u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
        } else {
            const uint4 a = __ldg(q);
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
        }
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            r.S[2 * k] = h(u[k], 0) * hd.x;
            r.S[2 * k + 1] = h(u[k], 1) * hd.x;
            r.chi[2 * k] = h(u[W / 2 + k], 0) * hd.y;
            r.chi[2 * k + 1] = h(u[W / 2 + k], 1) * hd.y;
        }
        return r;
    }
    __device__ __forceinline__ static void store(float* rec, const float* S, const float* chi)
    {
        float ms = 0.0f, mc = 0.0f;
#pragma unroll
        for (int w = 0; w < W; ++w) { ms = fmaxf(ms, S[w]); mc = fmaxf(mc, chi[w]); }
        if (!(ms > 0.0f)) ms = 1.0f;
        if (!(mc > 0.0f)) mc = 1.0f;
        unsigned int u[W];
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            u[k] = (unsigned int)__half_as_ushort(__float2half_rn(S[2 * k] / ms)) |
                   ((unsigned int)__half_as_ushort(__float2half_rn(S[2 * k + 1] / ms)) << 16);
            u[W / 2 + k] = (unsigned int)__half_as_ushort(__float2half_rn(chi[2 * k] / mc)) |
                           ((unsigned int)__half_as_ushort(__float2half_rn(chi[2 * k + 1] / mc)) << 16);
        }
        *reinterpret_cast<float4*>(rec) = make_float4(ms, mc, 0.0f, 0.0f);
        uint4* q = reinterpret_cast<uint4*>(rec + 4);
#pragma unroll
        for (int k = 0; k < W / 4; ++k) q[k] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
    }
};

// Layout of the 2D sparse grids' MIP bricks.  Level m of a block is side x side
// voxels (side = 16 >> m) stored row by row (z outer, x inner).  In float32 a
// row holds the S values of its voxels (W floats each, in x order) and then
// their chi values: rays of a warp at neighbouring voxels of a row read one
// contiguous run of S and one of chi, so a 256-bit warp load touches half as
// many 128-byte lines as with S and chi side by side per voxel (ncu on the
// 512^2 paired walk: L1 load wavefronts -30% for the same sectors).  The
// reduced-precision formats, whose records are 32 or 48 bytes, keep one record
// per voxel.
template <int W, int ST>
struct BrickFmt {
    static constexpr bool kSplit = ST == kStoreF32;
    static constexpr int kRec = RecFmt<W, ST>::kStride;  // floats per voxel
    static constexpr int kX = kSplit ? W : kRec;         // floats between x neighbours of a row
    // offset (floats) of voxel (lx, lz) of a level of `side` voxels per row whose
    // first voxel is voxel `first` of the brick array
    __host__ __device__ __forceinline__ static long long offset(long long first, int lz, int lx, int side)
    {
        return (first + (long long)lz * side) * kRec + (long long)lx * kX;
    }
    // floats from a voxel's S to its chi (0: a record holds both)
    __host__ __device__ __forceinline__ static int chi_off(int side) { return kSplit ? side * W : 0; }
    __device__ __forceinline__ static Record<W> load(const float* p, int coff)
    {
        if constexpr (kSplit) {
            Record<W> r;
            if constexpr (W == 8) {  // 32-byte aligned runs
                ldg256(p, r.S);
                ldg256(p + coff, r.chi);
            } else if constexpr (W == 4) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(p));
                const float4 c = __ldg(reinterpret_cast<const float4*>(p + coff));
                r.S[0] = a.x; r.S[1] = a.y; r.S[2] = a.z; r.S[3] = a.w;
                r.chi[0] = c.x; r.chi[1] = c.y; r.chi[2] = c.z; r.chi[3] = c.w;
            } else if constexpr (W == 2) {
                const float2 a = __ldg(reinterpret_cast<const float2*>(p));
                const float2 c = __ldg(reinterpret_cast<const float2*>(p + coff));
                r.S[0] = a.x; r.S[1] = a.y;
                r.chi[0] = c.x; r.chi[1] = c.y;
            } else {
                r.S[0] = __ldg(p);
                r.chi[0] = __ldg(p + coff);
            }
            return r;
        } else {
            return RecFmt<W, ST>::load(p);
        }
    }
    __device__ __forceinline__ static void store(float* p, int coff, const float* S, const float* chi)
    {
        if constexpr (kSplit) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                p[w] = S[w];
                p[coff + w] = chi[w];
            }
        } else {
            RecFmt<W, ST>::store(p, S, chi);
        }
    }
};

// Quadrature passed by value to the solve kernels.
struct Quadrature {
    int n_dir;
    float dx[DEX_MAX_DIRS];
    float dz[DEX_MAX_DIRS];
    float w[DEX_MAX_DIRS];
};

}  // namespace dex
