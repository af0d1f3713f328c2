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

cudaError_t measure_ex2_rate(cudaStream_t s, double* ops_per_s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = 8 * sms, threads = 256;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    if (e == cudaSuccess) {
        k_ex2_rate<<<blocks, threads, 0, s>>>(out, 64);  // warm-up
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, s);
            k_ex2_rate<<<blocks, threads, 0, s>>>(out, kProbeIters);
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
    if (e != cudaSuccess) return e;
    *ops_per_s = (double)blocks * threads * kProbeIters * kProbeChains / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace dex
