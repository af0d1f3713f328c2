// MIP chain construction and variance-limited level selection (Sections 2.1, 2.2, 2.3.1).
//
// One CTA per (active block, wavelength batch), one thread per MIP-0 cell of the
// 16 x 16 block.  Level m (voxel side Ds = 2^m) is built in shared memory from
// the 2 x 2 children of level m-1 for all W wavelengths of the batch:
//   value: geometric mean of the children (log-space mean, the default) or
//          their arithmetic mean (the box filter of Fig. 2);
//   test:  IoD[X] = |Var[X] / Mean[X]| (Eq. IoD) of X = ln(eta Ds) and
//          X = ln(chi Ds) over the 4 children, population variance; a group
//          passes if both IoDs are below their thresholds or if the largest
//          child chi times Ds is below chi_ds_min (the always-average rule).
// Children that mix zeros and non-zeros have no log mean: their value is the
// arithmetic mean and they pass only through the always-average rule.
// The block level is the largest m <= max_mip such that every group at every
// level <= m passes for every wavelength of the batch, optionally capped per
// block.  Every level of the chain is written as wavelength-batch records
// (S, chi) in the requested storage format (float32, stored per brick row as
// the row's S values then its chi values; bfloat16, or float16 with per-record
// scales, one record per voxel: BrickFmt); the level goes into the packed 3-bit
// state words (0 = empty, m + 1 = level m, 21 blocks per 64-bit word).
#include "vlm.cuh"

namespace dex {

namespace {

constexpr int kMaxLevels = 5;  // levels 0..4 of a 16 x 16 block

__host__ __device__ constexpr int level_offset(int m) { return 341 - (341 >> (2 * m)); }

// voxel (lx, lz) of the level of `side` voxels per row starting at voxel `first`
// of the block's chain `brick` (BrickFmt: float32 rows hold S, then chi)
template <int W, int ST>
__device__ __forceinline__ void store_record(float* brick, int first, int lz, int lx, int side, const float* e,
                                             const float* c)
{
    using BF = BrickFmt<W, ST>;
    float S[W], x[W];
#pragma unroll
    for (int w = 0; w < W; ++w) encode_voxel(e[w], c[w], S[w], x[w]);
    BF::store(brick + BF::offset(first, lz, lx, side), BF::chi_off(side), S, x);
}

template <int W, int ST>
__global__ void __launch_bounds__(256) k_mips_build(const MipParams P)
{
    constexpr int REC = RecFmt<W, ST>::kStride;
    // level m values: sm_e[level][w][voxel], voxel count (16 >> m)^2
    __shared__ float sm_e[level_offset(kMaxLevels)][W];
    __shared__ float sm_c[level_offset(kMaxLevels)][W];
    const int a = blockIdx.x;
    if (a >= *P.n_active) return;
    const int b = blockIdx.y;
    const int blk = P.active[a];
    const int bx = blk % P.nbx, bz = blk / P.nbx;
    const int t = threadIdx.x;
    const int x = bx * DEX_BLOCK + (t & 15), z = bz * DEX_BLOCK + (t >> 4);
    const long long c = (long long)z * P.nx + x;
    const long long n_cells = (long long)P.nx * P.nz;
    float* brick = P.bricks + ((size_t)b * P.cap_active + a) * P.chain * REC;

    // level 0
    {
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
        store_record<W, ST>(brick, 0, t >> 4, t & 15, DEX_BLOCK, e, x_);
    }
    __syncthreads();

    int level = 0;
    bool ok = true;
    for (int m = 1; m <= P.max_mip; ++m) {
        const int side = DEX_BLOCK >> m, side_p = side << 1;
        const int off = level_offset(m), off_p = level_offset(m - 1);
        const float ds = (float)(1 << m);
        const float ln_ds = (float)m * 0.69314718f;
        bool pass = true;
        if (t < side * side) {
            const int vx = t % side, vz = t / side;
            const int c0 = off_p + (2 * vz) * side_p + 2 * vx;
            float e[W], x_[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const GroupStat se = reduce_group(sm_e[c0][w], sm_e[c0 + 1][w], sm_e[c0 + side_p][w],
                                                  sm_e[c0 + side_p + 1][w], ln_ds, P.log_mean);
                const float k0 = sm_c[c0][w], k1 = sm_c[c0 + 1][w], k2 = sm_c[c0 + side_p][w],
                            k3 = sm_c[c0 + side_p + 1][w];
                const GroupStat sc = reduce_group(k0, k1, k2, k3, ln_ds, P.log_mean);
                const float kmax = fmaxf(fmaxf(k0, k1), fmaxf(k2, k3));
                const bool pw = (se.iod < P.thr_eta && sc.iod < P.thr_chi) || (kmax * ds < P.chi_ds_min);
                pass = pass && pw;
                e[w] = se.val;
                x_[w] = sc.val;
                sm_e[off + t][w] = se.val;
                sm_c[off + t][w] = sc.val;
            }
            store_record<W, ST>(brick, off, vz, vx, side, e, x_);
        }
        const int all = __syncthreads_and(pass ? 1 : 0);
        if (ok && all) level = m;
        else ok = false;
    }
    if (t == 0) {
        if (P.level_cap != nullptr) {
            const int cap = P.level_cap[blk];
            level = min(level, max(cap, 0));
        }
        const unsigned long long state = (unsigned long long)(level + 1);
        atomicOr(P.words + (size_t)b * P.n_words + blk / DEX_STATES_PER_WORD,
                 state << (DEX_STATE_BITS * (blk % DEX_STATES_PER_WORD)));
    }
}

}  // namespace

int chain_length(int max_mip) { return level_offset(max_mip + 1); }

cudaError_t launch_mips_build(cudaStream_t s, const MipParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(P.words, 0, sizeof(unsigned long long) * (size_t)P.n_words * P.n_batch, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    const int key = P.W * 4 + P.storage;
    switch (key) {
        case 1 * 4 + kStoreF32: k_mips_build<1, kStoreF32><<<grid, 256, 0, s>>>(P); break;
        case 2 * 4 + kStoreF32: k_mips_build<2, kStoreF32><<<grid, 256, 0, s>>>(P); break;
        case 4 * 4 + kStoreF32: k_mips_build<4, kStoreF32><<<grid, 256, 0, s>>>(P); break;
        case 8 * 4 + kStoreF32: k_mips_build<8, kStoreF32><<<grid, 256, 0, s>>>(P); break;
        case 4 * 4 + kStoreBF16: k_mips_build<4, kStoreBF16><<<grid, 256, 0, s>>>(P); break;
        case 8 * 4 + kStoreBF16: k_mips_build<8, kStoreBF16><<<grid, 256, 0, s>>>(P); break;
        case 4 * 4 + kStoreF16: k_mips_build<4, kStoreF16><<<grid, 256, 0, s>>>(P); break;
        case 8 * 4 + kStoreF16: k_mips_build<8, kStoreF16><<<grid, 256, 0, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dex
