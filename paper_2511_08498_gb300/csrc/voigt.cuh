// Voigt function H(a, x) = Re w(x + i a) on the GPU: the HUM1WEI24 form named in
// Section 3.2 (Schreier 2018), float32, with two changes for float32 conditioning.
//   |x| + a >= 15     : region I of Humlicek (1982), w = i z / (sqrt(pi) (z^2 - 1/2));
//   5 <= |x| + a < 15 : 8-term Laplace continued fraction (Gautschi 1970),
//                       w = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/...)));
//   |x| + a < 5, a >= 0.25 : Weideman (1994), N = 24,
//                   w = 2 p(Z) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
//                   Z = (L + i z) / (L - i z), p(Z) = sum_{n=1..24} a_n Z^(n-1);
//   |x| + a < 5, a < 0.25 : the Taylor series of w about the real axis,
//                   w(x + i a) = sum_n w^(n)(x) (i a)^n / n!, n <= 8, with
//                   w(x) = e^{-x^2} + i Im w(x) (Im w(x) = (2/sqrt(pi)) Dawson(x)
//                   from the Weideman sum at real z) and the derivatives from
//                   w' = -2 z w + 2 i / sqrt(pi), w^(n+1) = -2 z w^(n) - 2 n w^(n-1)
//                   (Abramowitz & Stegun 7.1.20); on the real axis the real and
//                   imaginary parts follow the same recurrence separately.
// Why: at small damping the line wing H ~ a / (sqrt(pi) x^2) is a small difference
// of O(0.05) real parts in Weideman's form, and in float32 the complex sum loses
// up to ~1e-3 of it (7.5e-4 at a = 1e-3, x ~ 3.9).  On the real axis only the
// imaginary part is taken from the sum, where nothing cancels; the real part is
// e^{-x^2} exactly, and the series in a needs no cancelling sum for a < 0.25.
// In float32 the whole evaluation stays within ~1e-5 relative of the Faddeeva
// function over the moving-medium workload's damping range (the continued
// fraction likewise replaces Weideman's sum for 5 <= |x| + a < 15, where it
// cancels as well).  The coefficients a_n (Fourier coefficients of
// exp(-t^2)(L^2 + t^2), t = L tan(theta/2)) are computed on the host and passed
// as a kernel parameter.
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
    if (a < 0.25f) {
        // w on the real axis at |x| (H is even in x): Z = (L + i x) / (L - i x)
        const float ax = fabsf(x);
        const float dd = __frcp_rn(fmaf(kWeidemanL, kWeidemanL, ax * ax));
        const float Zr = fmaf(kWeidemanL, kWeidemanL, -ax * ax) * dd;
        const float Zi = 2.0f * kWeidemanL * ax * dd;
        float pr = C.a[kWeidemanN - 1], pi = 0.0f;
#pragma unroll
        for (int n = kWeidemanN - 2; n >= 0; --n) {
            const float tr = fmaf(pr, Zr, fmaf(-pi, Zi, C.a[n]));
            pi = fmaf(pr, Zi, pi * Zr);
            pr = tr;
        }
        // 1 / (L - i x) = (L + i x) dd; Im of 2 p / (L - i x)^2 + 1 / (sqrt(pi) (L - i x))
        const float ir = kWeidemanL * dd, ii = ax * dd;
        const float i2r = ir * ir - ii * ii, i2i = 2.0f * ir * ii;
        // R_n, I_n: real and imaginary parts of w^(n)(x); term n of H is
        // Re[(i a)^n w^(n)] / n!: for n mod 4 = 0, 1, 2, 3 it is +R, -I, -R, +I
        float R0 = expf(-ax * ax);
        float I0 = 2.0f * fmaf(pr, i2i, pi * i2r) + kInvSqrtPi * ii;
        const float m2x = -2.0f * ax;
        float R1 = m2x * R0;
        float I1 = fmaf(m2x, I0, 2.0f * kInvSqrtPi);
        float h = R0;
        float c = a;  // a^n / n!
        h = fmaf(-c, I1, h);
#pragma unroll
        for (int n = 1; n < 8; ++n) {
            const float R2 = fmaf(m2x, R1, -2.0f * (float)n * R0);
            const float I2 = fmaf(m2x, I1, -2.0f * (float)n * I0);
            c *= a * (1.0f / (float)(n + 1));
            const int k = (n + 1) & 3;  // sign and part of term n + 1
            if (k == 0) h = fmaf(c, R2, h);
            else if (k == 1) h = fmaf(-c, I2, h);
            else if (k == 2) h = fmaf(-c, R2, h);
            else h = fmaf(c, I2, h);
            R0 = R1; R1 = R2;
            I0 = I1; I1 = I2;
        }
        return h;
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
