// Throughput of the special-function unit's 2^x (ex2.approx.ftz.f32), the one
// operation every segment-wavelength update needs: the ceiling the solve
// kernels are measured against.  Each thread runs 8 independent chains
// x <- 2^x * c (c = -1/2 keeps x in (-1, 0]); the grid fills every SM 8 times.
#include "dex_common.cuh"
#include "umma.cuh"

namespace dex {

namespace {

constexpr int kProbeIters = 4096;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) k_ex2_rate(float* out, int iters)
{
    float a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = -1e-3f * (float)(threadIdx.x + q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = ex2_approx(a[q]) * -0.5f;
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Throughput of the FP32 pipe on packed operations (FFMA2, two lane
// operations per instruction), the unit the update's multiplies and adds use:
// 8 independent chains a <- a * c + d per thread (c = 1 - 2^-10, d = 2^-10:
// a stays in [0, 1]).
__global__ void __launch_bounds__(256) k_fp32_rate(float* out, int iters)
{
    float2 a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = make_float2(1e-3f * (float)(threadIdx.x + q), 0.5f);
    const float2 c = make_float2(0.9990234375f, 0.9990234375f), d = make_float2(0.0009765625f, 0.0009765625f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = __ffma2_rn(a[q], c, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q].x + a[q].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// An mbarrier that nothing arrives on: the bounded wait every tensor-core
// kernel uses must give up after `polls` polls and report DEX_ERR_TIMEOUT,
// leaving the context usable.
__global__ void k_wait_timeout(int polls, unsigned int* status)
{
    __shared__ unsigned long long mbar;
    if (threadIdx.x == 0) umma::mbar_init(&mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !umma::mbar_wait(&mbar, 0u, polls)) raise_status(status, DEX_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_timeout(cudaStream_t s, int polls, unsigned int* status)
{
    k_wait_timeout<<<1, 32, 0, s>>>(polls, status);
    return cudaGetLastError();
}

// Best of 3 timed launches of a probe kernel (8 CTAs of 256 threads per SM,
// kProbeIters iterations of kProbeChains chains); returns the launch time in ms.
template <class K>
cudaError_t time_probe(cudaStream_t s, K kernel, int& blocks, float& best)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    blocks = 8 * sms;
    const int threads = 256;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    best = 0.0f;
    if (e == cudaSuccess) {
        kernel<<<blocks, threads, 0, s>>>(out, 64);  // warm-up
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, s);
            kernel<<<blocks, threads, 0, s>>>(out, kProbeIters);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return e;
}

cudaError_t measure_fp32_rate(cudaStream_t s, double* ops_per_s)
{
    int blocks = 0;
    float best = 0.0f;
    const cudaError_t e = time_probe(s, k_fp32_rate, blocks, best);
    if (e != cudaSuccess) return e;
    *ops_per_s = 2.0 * blocks * 256.0 * kProbeIters * kProbeChains / (best * 1e-3);
    return cudaSuccess;
}

cudaError_t measure_ex2_rate(cudaStream_t s, double* ops_per_s)
{
    int blocks = 0;
    float best = 0.0f;
    const cudaError_t e = time_probe(s, k_ex2_rate, blocks, best);
    if (e != cudaSuccess) return e;
    *ops_per_s = (double)blocks * 256.0 * kProbeIters * kProbeChains / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace dex
