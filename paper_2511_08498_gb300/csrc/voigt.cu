// Voigt function: host-side Weideman coefficients, constant-memory upload, and
// an elementwise kernel behind dex_voigt.
#include <cmath>
#include <mutex>

#include "dex_internal.h"
#include "voigt.cuh"

namespace dex {

namespace {

void weideman_coefficients(double* a, int n)
{
    const int M = 2 * n;
    const double L = std::sqrt(n / std::sqrt(2.0));
    for (int m = 1; m <= n; ++m) {
        double s = 0.0;
        for (int k = -M + 1; k <= M - 1; ++k) {  // theta = -pi contributes f = 0
            const double theta = k * M_PI / M;
            const double t = L * std::tan(theta / 2.0);
            s += std::exp(-t * t) * (L * L + t * t) * std::cos(m * theta);
        }
        a[m - 1] = s / (2.0 * M);
    }
}

__global__ void k_voigt(const VoigtCoef C, long long n, const float* __restrict__ a, const float* __restrict__ x,
                        float* __restrict__ h)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        h[i] = voigt_h(C, a[i], x[i]);
}

}  // namespace

const VoigtCoef& voigt_coefficients()
{
    static VoigtCoef coef;
    static std::once_flag once;
    std::call_once(once, [] {
        double a[kWeidemanN];
        weideman_coefficients(a, kWeidemanN);
        for (int i = 0; i < kWeidemanN; ++i) coef.a[i] = (float)a[i];
    });
    return coef;
}

cudaError_t launch_voigt(cudaStream_t s, long long n, const float* a, const float* x, float* h)
{
    if (n == 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    k_voigt<<<(unsigned)b, 256, 0, s>>>(voigt_coefficients(), n, a, x, h);
    return cudaGetLastError();
}

}  // namespace dex
