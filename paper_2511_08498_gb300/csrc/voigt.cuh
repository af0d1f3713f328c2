// Voigt function H(a, x) = Re w(x + i a) on the GPU: the HUM1WEI24 form named in
// Section 3.2 (Schreier 2018), float32, with one change for float32 conditioning.
//   |x| + a >= 15     : region I of Humlicek (1982), w = i z / (sqrt(pi) (z^2 - 1/2));
//   5 <= |x| + a < 15 : 8-term Laplace continued fraction (Gautschi 1970),
//                       w = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/...)));
//                       in float32 the Weideman sum below cancels O(1) terms down
//                       to H ~ 1e-5 there (errors up to ~1e-3), the fraction does not;
//   |x| + a < 5       : Weideman (1994), N = 24,
//                   w = 2 p(Z) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
//                   Z = (L + i z) / (L - i z), p(Z) = sum_{n=1..24} a_n Z^(n-1).
// The coefficients a_n (Fourier coefficients of exp(-t^2)(L^2 + t^2),
// t = L tan(theta/2)) are computed on the host and passed as a kernel parameter.
#pragma once

#include <cuda_runtime.h>

namespace dex {

constexpr int kWeidemanN = 24;
constexpr float kWeidemanL = 4.1195342878f;         // sqrt(24 / sqrt 2)
constexpr float kInvSqrtPi = 0.56418958354775628f;

struct VoigtCoef {
    float a[kWeidemanN];  // a_1 .. a_24
};

// Host: the coefficients, computed once in double from the definition
// (trapezoid rule on 4N points) and rounded to float.
const VoigtCoef& voigt_coefficients();

__device__ __forceinline__ float voigt_h(const VoigtCoef& C, float a, float x)
{
    const float s = fabsf(x) + a;
    if (s >= 5.0f && s < 15.0f) {
        // f = z - (k/2) / f, innermost k = 8; w = (i / sqrt(pi)) / f -> Re w = Im f / (sqrt(pi) |f|^2)
        float fr = x, fi = a;
#pragma unroll
        for (int k = 8; k >= 1; --k) {
            const float c = 0.5f * (float)k;
            const float q = __fdividef(c, fmaf(fr, fr, fi * fi));
            fr = fmaf(-q, fr, x);
            fi = fmaf(q, fi, a);
        }
        return kInvSqrtPi * __fdividef(fi, fmaf(fr, fr, fi * fi));
    }
    if (s >= 15.0f) {
        // i z / (sqrt(pi) (z^2 - 1/2)), z = x + i a
        const float zr = x, zi = a;
        const float dr = zr * zr - zi * zi - 0.5f, di = 2.0f * zr * zi;   // z^2 - 1/2
        const float nr = -zi, ni = zr;                                     // i z
        const float inv = __fdividef(1.0f, dr * dr + di * di);
        return kInvSqrtPi * (nr * dr + ni * di) * inv;                     // Re(n / d)
    }
    // den = L - i z = (L + a) - i x ; num = L + i z = (L - a) + i x
    const float denr = kWeidemanL + a, deni = -x;
    const float numr = kWeidemanL - a, numi = x;
    // correctly rounded: a 2-ulp reciprocal would be amplified by the cancelling sum
    const float dd = __frcp_rn(fmaf(denr, denr, deni * deni));
    // Z = num / den
    const float Zr = (numr * denr + numi * deni) * dd;
    const float Zi = (numi * denr - numr * deni) * dd;
    float pr = C.a[kWeidemanN - 1], pi = 0.0f;
#pragma unroll
    for (int n = kWeidemanN - 2; n >= 0; --n) {  // Horner
        const float tr = fmaf(pr, Zr, fmaf(-pi, Zi, C.a[n]));
        pi = fmaf(pr, Zi, pi * Zr);
        pr = tr;
    }
    // 1 / den and 1 / den^2
    const float ir = denr * dd, ii = -deni * dd;
    const float i2r = ir * ir - ii * ii, i2i = 2.0f * ir * ii;
    return 2.0f * (pr * i2r - pi * i2i) + kInvSqrtPi * ir;
}

}  // namespace dex
