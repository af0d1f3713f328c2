// The 3D adapted grid (Section 2.3: cubic 8^3 blocks, one refinement level per
// block, at most level 3 so that a block reduces to one voxel; Section 2.1:
// volumetric MIPs over 2x2x2 voxels): the block sparsity map, the Morton-ordered
// block layout, and the MIP chains with the variance-limited level choice.
//
// Grid [nz][ny][nx], x fastest.  Block (bx, by, bz) has index
// (bz * nby + by) * nbx + bx; its Morton code interleaves bx, by, bz into bits
// 3b, 3b + 1, 3b + 2.  A chain stores level m as (8 >> m)^3 records, row-major
// [z][y][x], after the (8 >> k)^3 records of every finer level k < m.
#include "vlm.cuh"

namespace dex {

namespace {

constexpr int B3 = DEX_BLOCK3;
constexpr int kCells3 = B3 * B3 * B3;  // 512

__host__ __device__ constexpr int level_offset3(int m) { return 585 - (585 >> (3 * m)); }

// flag[blk] = 1 if any cell of the block has eta != 0 or chi != 0 at any wavelength
__global__ void __launch_bounds__(kCells3) k_block_flags3(int nx, int ny, int nbx, int nby, long long n_cells,
                                                          int n_lambda, const float* __restrict__ eta,
                                                          const float* __restrict__ chi, int* __restrict__ flag)
{
    const int blk = blockIdx.x;
    const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
    const int t = threadIdx.x;
    const int x = bx * B3 + (t & 7), y = by * B3 + ((t >> 3) & 7), z = bz * B3 + (t >> 6);
    const long long c = ((long long)z * ny + y) * nx + x;
    int any = 0;
    for (int l = 0; l < n_lambda && !any; ++l)
        any = (eta[l * n_cells + c] != 0.0f) | (chi[l * n_cells + c] != 0.0f);
    any = __syncthreads_or(any);
    if (t == 0) flag[blk] = any ? 1 : 0;
}

// every third bit of v, packed (inverse of the 3-way bit interleave)
__device__ __forceinline__ unsigned compact1by2(unsigned v)
{
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030c30c3u;
    v = (v ^ (v >> 4)) & 0x0300f00fu;
    v = (v ^ (v >> 8)) & 0xff0000ffu;
    v = (v ^ (v >> 16)) & 0x000003ffu;
    return v;
}

// One CTA walks the Z-order curve over a P^3 cube of blocks (P = power of two
// >= every block extent); non-empty blocks get consecutive ranks.  offset[]
// holds the flags on entry and the ranks (or -1) on exit.
__global__ void __launch_bounds__(1024) k_block_layout3(int nbx, int nby, int nbz, int log2P,
                                                        int* __restrict__ offset, int* __restrict__ active,
                                                        int* __restrict__ n_active)
{
    __shared__ int scan[1024];
    const unsigned total = 1u << (3 * log2P);
    const unsigned per = (total + blockDim.x - 1) / blockDim.x;
    const unsigned lo = threadIdx.x * per, hi = min(total, lo + per);
    int cnt = 0;
    for (unsigned code = lo; code < hi; ++code) {
        const int bx = (int)compact1by2(code), by = (int)compact1by2(code >> 1), bz = (int)compact1by2(code >> 2);
        if (bx < nbx && by < nby && bz < nbz) cnt += offset[(bz * nby + by) * nbx + bx] != 0;
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
        const int bx = (int)compact1by2(code), by = (int)compact1by2(code >> 1), bz = (int)compact1by2(code >> 2);
        if (bx < nbx && by < nby && bz < nbz) {
            const int blk = (bz * nby + by) * nbx + bx;
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

template <int W, int ST>
__device__ __forceinline__ void store_record3(float* rec, const float* e, const float* c)
{
    float S[W], x[W];
#pragma unroll
    for (int w = 0; w < W; ++w) encode_voxel(e[w], c[w], S[w], x[w]);
    RecFmt<W, ST>::store(rec, S, x);
}

// One CTA per (active block, wavelength batch), one thread per MIP-0 cell.
// Level m is formed in shared memory from the 2x2x2 children of level m-1 for
// the W wavelengths of the batch (value: log-space or box-filter mean; test:
// IoD of ln(eta Ds) and ln(chi Ds) below their thresholds, or the largest child
// chi times Ds below chi_ds_min).  The block level is the largest m such that
// every group of every level <= m passes for every wavelength of the batch.
template <int W, int ST>
__global__ void __launch_bounds__(kCells3) k_mips3_build(const Mip3Params P)
{
    constexpr int REC = RecFmt<W, ST>::kStride;
    __shared__ float sm_e[level_offset3(4)][W];
    __shared__ float sm_c[level_offset3(4)][W];
    const int a = blockIdx.x;
    if (a >= *P.n_active) return;
    const int b = blockIdx.y;
    const int blk = P.active[a];
    const int bx = blk % P.nbx, by = (blk / P.nbx) % P.nby, bz = blk / (P.nbx * P.nby);
    const int t = threadIdx.x;
    const int x = bx * B3 + (t & 7), y = by * B3 + ((t >> 3) & 7), z = bz * B3 + (t >> 6);
    const long long c = ((long long)z * P.ny + y) * P.nx + x;
    const long long n_cells = (long long)P.nx * P.ny * P.nz;
    float* brick = P.bricks + ((size_t)b * P.cap_active + a) * P.chain * REC;

    {  // level 0
        float e[W], x_[W];
        bool bad = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int l = b * W + w;
            float ev = 0.0f, cv = 0.0f;
            if (l < P.n_lambda) {
                ev = P.eta[l * n_cells + c];
                cv = P.chi[l * n_cells + c];
                if (!(ev >= 0.0f) || !(cv >= 0.0f) || !isfinite(ev) || !isfinite(cv) ||
                    (cv == 0.0f && ev > kEmitterMaxEta)) {
                    bad = true;
                    ev = cv = 0.0f;
                }
            }
            e[w] = ev;
            x_[w] = cv;
            sm_e[t][w] = ev;
            sm_c[t][w] = cv;
        }
        if (bad) raise_status(P.status, DEX_ERR_NUMERIC);
        store_record3<W, ST>(brick + (size_t)t * REC, e, x_);
    }
    __syncthreads();

    int level = 0;
    bool ok = true;
    for (int m = 1; m <= P.max_mip; ++m) {
        const int side = B3 >> m, sp = side << 1, sp2 = sp * sp;
        const int off = level_offset3(m), off_p = level_offset3(m - 1);
        const float ds = (float)(1 << m);
        const float ln_ds = (float)m * 0.69314718f;
        bool pass = true;
        if (t < side * side * side) {
            const int vx = t % side, vy = (t / side) % side, vz = t / (side * side);
            const int c0 = off_p + ((2 * vz) * sp + 2 * vy) * sp + 2 * vx;
            const int kid[8] = {c0, c0 + 1, c0 + sp, c0 + sp + 1, c0 + sp2, c0 + sp2 + 1, c0 + sp2 + sp,
                                c0 + sp2 + sp + 1};
            float e[W], x_[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                float ge[8], gc[8];
                float kmax = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    ge[q] = sm_e[kid[q]][w];
                    gc[q] = sm_c[kid[q]][w];
                    kmax = fmaxf(kmax, gc[q]);
                }
                const GroupStat se = reduce_group8(ge, ln_ds, P.log_mean);
                const GroupStat sc = reduce_group8(gc, ln_ds, P.log_mean);
                const bool pw = (se.iod < P.thr_eta && sc.iod < P.thr_chi) || (kmax * ds < P.chi_ds_min);
                pass = pass && pw;
                e[w] = se.val;
                x_[w] = sc.val;
                sm_e[off + t][w] = se.val;
                sm_c[off + t][w] = sc.val;
            }
            store_record3<W, ST>(brick + (size_t)(off + t) * REC, e, x_);
        }
        const int all = __syncthreads_and(pass ? 1 : 0);
        if (ok && all) level = m;
        else ok = false;
    }
    if (t == 0) {
        if (P.level_cap != nullptr) level = min(level, max((int)P.level_cap[blk], 0));
        const unsigned long long state = (unsigned long long)(level + 1);
        atomicOr(P.words + (size_t)b * P.n_words + blk / DEX_STATES_PER_WORD,
                 state << (DEX_STATE_BITS * (blk % DEX_STATES_PER_WORD)));
    }
}

}  // namespace

int chain_length3(int max_mip) { return level_offset3(max_mip + 1); }

cudaError_t launch_grid3_build(cudaStream_t s, int nx, int ny, int nz, int n_lambda, const float* eta,
                               const float* chi, int* block_offset, int* active, int* n_active)
{
    const int nbx = nx / B3, nby = ny / B3, nbz = nz / B3;
    const long long n_cells = (long long)nx * ny * nz;
    k_block_flags3<<<(unsigned)(nbx * nby * nbz), kCells3, 0, s>>>(nx, ny, nbx, nby, n_cells, n_lambda, eta, chi,
                                                                   block_offset);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int log2P = 0;
    while ((1 << log2P) < nbx || (1 << log2P) < nby || (1 << log2P) < nbz) ++log2P;
    k_block_layout3<<<1, 1024, 0, s>>>(nbx, nby, nbz, log2P, block_offset, active, n_active);
    return cudaGetLastError();
}

cudaError_t launch_mips3_build(cudaStream_t s, const Mip3Params& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(P.words, 0, sizeof(unsigned long long) * (size_t)P.n_words * P.n_batch, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    switch (P.W * 4 + P.storage) {
        case 1 * 4 + kStoreF32: k_mips3_build<1, kStoreF32><<<grid, kCells3, 0, s>>>(P); break;
        case 2 * 4 + kStoreF32: k_mips3_build<2, kStoreF32><<<grid, kCells3, 0, s>>>(P); break;
        case 4 * 4 + kStoreF32: k_mips3_build<4, kStoreF32><<<grid, kCells3, 0, s>>>(P); break;
        case 8 * 4 + kStoreF32: k_mips3_build<8, kStoreF32><<<grid, kCells3, 0, s>>>(P); break;
        case 4 * 4 + kStoreBF16: k_mips3_build<4, kStoreBF16><<<grid, kCells3, 0, s>>>(P); break;
        case 8 * 4 + kStoreBF16: k_mips3_build<8, kStoreBF16><<<grid, kCells3, 0, s>>>(P); break;
        case 4 * 4 + kStoreF16: k_mips3_build<4, kStoreF16><<<grid, kCells3, 0, s>>>(P); break;
        case 8 * 4 + kStoreF16: k_mips3_build<8, kStoreF16><<<grid, kCells3, 0, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dex
