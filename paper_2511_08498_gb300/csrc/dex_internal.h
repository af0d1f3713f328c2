// Internal launch interfaces between the C-ABI layer (dex_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dex_common.cuh"

namespace dex {

struct DenseParams {
    int nx, nz, n_lambda, W, n_batch;
    long long n_cells;
    const float* planes;
    int n_probe;
    const int* probes;      // nullptr: every cell, tiled launch
    float i_bc;
    float* J;
    float* I;
    unsigned long long* seg_count;
    unsigned int* status;
    Quadrature quad;
};

cudaError_t launch_pack_planes(cudaStream_t s, long long n_cells, int n_lambda, int W,
                               const float* eta, const float* chi, float* planes, unsigned int* status);
cudaError_t launch_solve_dense(cudaStream_t s, const DenseParams& p);

}  // namespace dex
