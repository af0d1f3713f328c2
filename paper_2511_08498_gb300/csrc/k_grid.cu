// MIP-0 emissivity/opacity of the static continuum + line model, the block
// sparsity map and the Morton-ordered block layout (Sections 2 and 2.3.1).
#include "dex_internal.h"

namespace dex {

namespace {

// Eqs. EtaTot/ChiTot for one line plus a continuum background:
//   chi_l = ratio * chi_c * exp(-(dlam / dld)^2), chi = chi_c + chi_l,
//   eta = chi_c S_c + chi_l S_l.
__global__ void k_synth_static_line(long long n_cells, int n_lambda, const float* __restrict__ chi_c,
                                    const float* __restrict__ s_c, const float* __restrict__ s_l,
                                    const float* __restrict__ ratio, const float* __restrict__ dld,
                                    const float* __restrict__ dlam, float* __restrict__ eta,
                                    float* __restrict__ chi)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const float cc = chi_c[c], sc = s_c[c], sl = s_l[c], r = ratio[c], inv_w = 1.0f / dld[c];
        const float ec = cc * sc, rc = r * cc;
        for (int l = 0; l < n_lambda; ++l) {
            const float u = dlam[l] * inv_w;
            const float cl = rc * expf(-u * u);
            chi[(long long)l * n_cells + c] = cc + cl;
            eta[(long long)l * n_cells + c] = fmaf(cl, sl, ec);
        }
    }
}

// flag[blk] = 1 if any cell of the block has eta != 0 or chi != 0 at any wavelength
__global__ void __launch_bounds__(256) k_block_flags(int nx, int nbx, long long n_cells, int n_lambda,
                                                     const float* __restrict__ eta,
                                                     const float* __restrict__ chi, int* __restrict__ flag)
{
    const int blk = blockIdx.x;
    const int bx = blk % nbx, bz = blk / nbx;
    const int x = bx * DEX_BLOCK + (threadIdx.x & 15), z = bz * DEX_BLOCK + (threadIdx.x >> 4);
    const long long c = (long long)z * nx + x;
    int any = 0;
    for (int l = 0; l < n_lambda && !any; ++l)
        any = (eta[l * n_cells + c] != 0.0f) | (chi[l * n_cells + c] != 0.0f);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) flag[blk] = any ? 1 : 0;
}

__device__ __forceinline__ unsigned compact1by1(unsigned v)
{
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}

// One CTA: walk the Z-order curve over a P x P block square (P = power of two
// >= max(nbx, nbz)); non-empty blocks get consecutive ranks.  offset[] holds
// the flags on entry and the ranks (or -1) on exit; active[rank] = block index.
__global__ void __launch_bounds__(1024) k_block_layout(int nbx, int nbz, int log2P, int* __restrict__ offset,
                                                       int* __restrict__ active, int* __restrict__ n_active)
{
    __shared__ int scan[1024];
    const unsigned total = 1u << (2 * log2P);
    const unsigned per = (total + blockDim.x - 1) / blockDim.x;
    const unsigned lo = threadIdx.x * per, hi = min(total, lo + per);
    int cnt = 0;
    for (unsigned code = lo; code < hi; ++code) {
        const int bx = (int)compact1by1(code), bz = (int)compact1by1(code >> 1);
        if (bx < nbx && bz < nbz) cnt += offset[bz * nbx + bx] != 0;
    }
    scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive Hillis-Steele scan
        const int v = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    int rank = scan[threadIdx.x] - cnt;
    for (unsigned code = lo; code < hi; ++code) {
        const int bx = (int)compact1by1(code), bz = (int)compact1by1(code >> 1);
        if (bx < nbx && bz < nbz) {
            const int blk = bz * nbx + bx;
            if (offset[blk] != 0) {
                active[rank] = blk;
                offset[blk] = rank++;
            } else {
                offset[blk] = -1;
            }
        }
    }
    if (threadIdx.x == blockDim.x - 1) *n_active = scan[threadIdx.x];
}

}  // namespace

cudaError_t launch_synth_static_line(cudaStream_t s, long long n_cells, int n_lambda, const float* chi_c,
                                     const float* s_c, const float* s_l, const float* ratio, const float* dld,
                                     const float* dlam, float* eta, float* chi)
{
    if (n_cells == 0 || n_lambda == 0) return cudaSuccess;
    long long blocks = (n_cells + 255) / 256;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    k_synth_static_line<<<(unsigned)blocks, 256, 0, s>>>(n_cells, n_lambda, chi_c, s_c, s_l, ratio, dld, dlam,
                                                         eta, chi);
    return cudaGetLastError();
}

cudaError_t launch_grid_build(cudaStream_t s, int nx, int nz, int n_lambda, const float* eta, const float* chi,
                              int* block_offset, int* active, int* n_active)
{
    const int nbx = nx / DEX_BLOCK, nbz = nz / DEX_BLOCK;
    const long long n_cells = (long long)nx * nz;
    k_block_flags<<<(unsigned)(nbx * nbz), 256, 0, s>>>(nx, nbx, n_cells, n_lambda, eta, chi, block_offset);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_block_layout(s, nbx, nbz, block_offset, active, n_active);
}

cudaError_t launch_block_layout(cudaStream_t s, int nbx, int nbz, int* block_offset, int* active, int* n_active)
{
    int log2P = 0;
    while ((1 << log2P) < nbx || (1 << log2P) < nbz) ++log2P;
    k_block_layout<<<1, 1024, 0, s>>>(nbx, nbz, log2P, block_offset, active, n_active);
    return cudaGetLastError();
}

}  // namespace dex
