// Hierarchical DDA formal solver with one walk per ray for a pair of
// wavelength batches (Section 2.3, Algorithm 1 with Section 2.3.1; Section
// 4.1's wavelength batches and distance limits; Eq. RteIntegral per segment).
//
// The per-batch solver (k_hdda.cu) traces every ray once per batch of 8
// wavelengths, and about two thirds of its instructions are the walk: plane
// arithmetic, block crossings and level look-ups.  Here one thread carries the
// 16 wavelengths of two batches along one walk and integrates both batches'
// records of every voxel it leaves.  The batches pair mirror-wise within
// consecutive groups (pair_batches: b with n_batch - 1 - b for one group of all
// batches; a line's own batches when each group is one line's samples).  A
// line's batches lie symmetrically about its centre, so the two batches of a
// pair see the same part of the profile and tend to take the same levels (on
// the benchmark's static-line atmosphere every block's levels agree); the walk
// uses, in every block, the smaller of the two levels (Section 2.2), capped by
// the distance limits as usual.  No batch is integrated more coarsely than at
// its own levels.
//
// The walk and the update are those of k_solve_hdda_t (trace_ray) with a
// two-record voxel model; J and I equal, bit for bit, those of the per-batch
// walk given state words that hold the pair's minimum for both batches.  The
// middle batch of a group of odd size is solved by the per-batch walk.
#include "hdda.cuh"

namespace dex {

namespace {

// Launch shape per brick format.  The pair's state (16 intensities and
// transmissions, two records loaded at the top of each step) takes about 125
// registers with float32 records: 2 CTAs of 256 threads per SM.  Bfloat16
// records hold half the registers and run at 5 CTAs of 128 threads (at most 102
// registers).  Measured on the 1024^2 static-line solve (IoD 1e-2 / unlimited
// averaging), float32 on brick rows:
//   float32, 256 threads, 2 CTAs (this)          158.8 / 63.3 ms
//   float32, 128 threads, 4 CTAs                 167.1 / 66.8 ms
//   float32, 128 threads, 3 CTAs (160 registers) 168.0 / 67.5 ms
//   float32, 64 threads, 8 CTAs                  167.6 / 67.4 ms
//   float32, 256 threads, 1 CTA (194 registers)  204.5 / 82.0 ms
// with float32 records of S and chi side by side (before the brick rows):
//   float32, 256 threads, 2 CTAs                 173.6 / 62.8 ms
//   float32, 128 threads, 5 CTAs (96 registers)  176.4 / 66.1 ms
//   float32, 256 threads, 3 CTAs (80, spills)    294.4 / 106.1 ms
//   bfloat16, 128 threads, 5 CTAs (this)         165.0 / 66.2 ms
//   bfloat16, 256 threads, 2 CTAs                171.5 / 66.6 ms
//   bfloat16, 128 threads, 6 CTAs (80 registers) 174.3 / 69.8 ms
// and, for float32 at 256 threads, the step loop unrolled twice or not at all
// +1.4%, records loaded after the stepping +3.7%.
template <int ST>
constexpr int pair_threads() { return ST == kStoreBF16 ? 128 : 256; }
template <int ST>
constexpr int pair_min_blocks() { return ST == kStoreBF16 ? 5 : 2; }
// probes per CTA: 16 x (threads / 16) rows of a block; CTAs per active block and pair
template <int ST>
constexpr int pair_parts() { return DEX_BLOCK * DEX_BLOCK / pair_threads<ST>(); }

template <int ST>
using PairModel = PairRecModel<ST, pair_min_blocks<ST>()>;

// EXT: each probe's own-voxel emission is left out (the first segment of every
// ray, as k_solve_hdda_t with EXT).
template <int ST, bool COUNT, bool EXT>
__global__ void __launch_bounds__(pair_threads<ST>(), pair_min_blocks<ST>()) k_solve_hdda_pair(const HddaParams P)
{
    using Model = PairModel<ST>;
    constexpr int kParts = pair_parts<ST>();
    extern __shared__ int s_info[];
    __shared__ float s_J[16][pair_threads<ST>()];
    __shared__ int s_box[4];
    const int a0 = blockIdx.x / kParts, part = blockIdx.x - a0 * kParts;
    if (a0 >= *P.n_active) return;
    int b1, b2;
    pair_batches(blockIdx.y, P.n_batch, P.pair_group, b1, b2);
    const int tid = threadIdx.x;
    const unsigned long long* w1 = P.words + (size_t)b1 * P.n_words;
    const unsigned long long* w2 = P.words + (size_t)b2 * P.n_words;
    const int n_blocks = P.nbx * P.nbz;
    for (int q = tid; q < n_blocks; q += blockDim.x)
        s_info[q] = pack_block_info(P.block_offset[q], min(block_state(w1, q), block_state(w2, q)));
#pragma unroll
    for (int w = 0; w < 16; ++w) s_J[w][tid] = 0.0f;
    if (tid < 4) s_box[tid] = (tid & 1) ? -1 : 0x7fffffff;
    __syncthreads();
    {
        // box around the non-empty blocks, in block units
        int xlo = 0x7fffffff, xhi = -1, zlo = 0x7fffffff, zhi = -1;
        const int na = *P.n_active;
        for (int q = tid; q < na; q += blockDim.x) {
            const int blk = P.active[q];
            const int bz = blk / P.nbx, bx = blk - bz * P.nbx;
            xlo = min(xlo, bx);
            xhi = max(xhi, bx);
            zlo = min(zlo, bz);
            zhi = max(zhi, bz);
        }
        xlo = __reduce_min_sync(0xffffffffu, xlo);
        xhi = __reduce_max_sync(0xffffffffu, xhi);
        zlo = __reduce_min_sync(0xffffffffu, zlo);
        zhi = __reduce_max_sync(0xffffffffu, zhi);
        if ((tid & 31) == 0) {
            atomicMin(&s_box[0], xlo);
            atomicMax(&s_box[1], xhi);
            atomicMin(&s_box[2], zlo);
            atomicMax(&s_box[3], zhi);
        }
    }
    __syncthreads();

    const int blk0 = P.active[a0];
    const int bx0 = blk0 % P.nbx, bz0 = blk0 / P.nbx;
    // the CTA's probes: rows part * (16 / kParts) .. of the block; warp w covers an
    // 8 x 4 tile of them (as in k_solve_hdda_t)
    const int wrp = tid >> 5;
    const int i = bx0 * DEX_BLOCK + (wrp & 1) * 8 + (tid & 7);
    const int j = bz0 * DEX_BLOCK + part * (DEX_BLOCK / kParts) + (wrp >> 1) * 4 + ((tid & 31) >> 3);
    const int state0 = (s_info[blk0] & 7) - 1;
    if (state0 < 0) {  // state words do not describe this active block
        raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
        return;
    }
    const size_t batch_floats = (size_t)P.cap_active * P.chain * Model::kStride;
    Geo G;
    G.nx = P.nx;
    G.nz = P.nz;
    G.nbx = P.nbx;
    G.nbz = P.nbz;
    G.chain = P.chain;
    G.cap_active = P.cap_active;
    G.batch_base = P.bricks + (size_t)b1 * batch_floats;
    G.x_lo = s_box[0] * DEX_BLOCK;
    G.x_hi = (s_box[1] + 1) * DEX_BLOCK;
    G.z_lo = s_box[2] * DEX_BLOCK;
    G.z_hi = (s_box[3] + 1) * DEX_BLOCK;
#pragma unroll
    for (int q = 0; q < 4; ++q) G.band[q] = P.band[q];
    const typename Model::Params M{(long long)(b2 - b1) * (long long)batch_floats};
    const int mip0 = min(state0, distance_cap(G, 0.0f));
    unsigned int nseg = 0;
    bool capped = false;

    for (int k = 0; k < P.quad.n_dir; ++k) {
        const float dx = P.quad.dx[k], dz = P.quad.dz[k];
        float I[16], T[16];
#pragma unroll
        for (int w = 0; w < 16; ++w) {
            I[w] = 0.0f;
            T[w] = 1.0f;
        }
        trace_ray<16, COUNT, Model, InfoLookup, EXT>(G, M, b1, i, j, bx0, bz0, a0, mip0, dx, dz, InfoLookup{s_info},
                                                     I, T, nseg, capped);
        const float wk = P.quad.w[k];
#pragma unroll
        for (int w = 0; w < 16; ++w) {
            const float Iw = fmaf(T[w], P.i_bc, I[w]);
            s_J[w][tid] = fmaf(wk, Iw, s_J[w][tid]);
            const int l = w < 8 ? b1 * 8 + w : b2 * 8 + (w - 8);
            if (P.I != nullptr && l < P.n_lambda)
                P.I[((size_t)l * P.quad.n_dir + k) * P.n_cells + (size_t)j * P.nx + i] = Iw;
        }
    }
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        const int l = w < 8 ? b1 * 8 + w : b2 * 8 + (w - 8);
        if (l < P.n_lambda) P.J[(size_t)l * P.n_cells + (size_t)j * P.nx + i] = s_J[w][tid];
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    // segments of the two batches
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, 2ull * nseg);
}

template <int ST>
cudaError_t launch_pair(cudaStream_t s, const HddaParams& P)
{
    const size_t smem = sizeof(int) * (size_t)P.nbx * P.nbz;
    dim3 grid((unsigned)(P.cap_active * pair_parts<ST>()), (unsigned)pair_count(P.n_batch, P.pair_group));
    auto kernel = P.exclude_own ? (P.seg_count ? k_solve_hdda_pair<ST, true, true> : k_solve_hdda_pair<ST, false, true>)
                                : (P.seg_count ? k_solve_hdda_pair<ST, true, false> : k_solve_hdda_pair<ST, false, false>);
    if (smem > 24 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, pair_threads<ST>(), smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

bool solve_hdda_paired_applies(const HddaParams& P)
{
    const long long n_blocks = (long long)P.nbx * P.nbz;
    return P.traversal == DEX_TRAVERSAL_PAIRED && P.W == 8 && n_blocks <= kPairInfoMaxBlocks &&
           (!P.exclude_own || P.storage == kStoreF32);
}

cudaError_t launch_solve_hdda_paired(cudaStream_t s, const HddaParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    if (pair_count(P.n_batch, P.pair_group) > 0) {
        cudaError_t e;
        switch (P.storage) {
            case kStoreF32: e = launch_pair<kStoreF32>(s, P); break;
            case kStoreBF16: e = launch_pair<kStoreBF16>(s, P); break;
            case kStoreF16: e = launch_pair<kStoreF16>(s, P); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    // the middle batch of every group of odd size alone, by the per-batch walk on
    // a view of that batch
    for (int q = 0; q < pair_lone_count(P.n_batch, P.pair_group); ++q) {
        const int m = pair_lone_batch(q, P.n_batch, P.pair_group);
        HddaParams Q = P;
        Q.traversal = DEX_TRAVERSAL_PER_BATCH;
        Q.n_batch = 1;
        Q.n_lambda = min(8, P.n_lambda - m * 8);
        Q.bricks = P.bricks + (size_t)m * P.cap_active * P.chain * record_floats(8, P.storage);
        Q.words = P.words + (size_t)m * P.n_words;
        Q.J = P.J + (size_t)m * 8 * P.n_cells;
        Q.I = P.I ? P.I + (size_t)m * 8 * P.quad.n_dir * P.n_cells : nullptr;
        if (cudaError_t e = launch_solve_hdda(s, Q)) return e;
    }
    return cudaSuccess;
}

}  // namespace dex
