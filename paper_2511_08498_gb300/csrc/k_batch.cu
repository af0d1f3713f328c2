// Many independent atmospheres in one persistent launch.
//
// Work items are (atmosphere, wavelength batch, active block, part of the
// block), numbered atmosphere by atmosphere (item_base[a] + (batch * capacity_a
// + rank) * parts + part).  A fixed grid of CTAs pulls `chunk` items at a time
// from a device counter (the queue) until it runs dry; each item is the block
// solve of k_solve_hdda_t (shared trace_ray) over 256 / parts of its probes.  Consecutive items mostly share an atmosphere and batch, so the
// staged block states and quadrature are reused, and the L2 working set stays
// one atmosphere batch wide.  Per-atmosphere completion times (globaltimer, ns)
// are recorded when requested.

#include "hdda.cuh"

namespace dex {

namespace {

// Scratch of the allocation-free entry point (dex_batch_solve_noalloc): a
// statically sized device array, present on every GPU that loads the library
// until the process exits.  Word 0 is the work counter.  Calls that overlap on
// the GPU share it and race.
static __device__ __align__(256) unsigned int g_noalloc_scratch[DEX_NOALLOC_SCRATCH_WORDS];

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int W>
struct StaticRec {
    static constexpr int kStride = 2 * W;
    static constexpr bool kSplit = true;  // float32 brick rows: S of the row, then chi
    static constexpr int kSplitStride = W;
    static constexpr bool kEarlyLoad = true;  // as the float32 static model of the single-grid solve
    static constexpr bool kZeroNoop = true;
    struct Params {
        int unused;
    };
    using Voxel = Record<W>;
    __device__ __forceinline__ static Voxel load_split(const Params&, const float* p, int coff)
    {
        return BrickFmt<W, kStoreF32>::load(p, coff);
    }
    __device__ __forceinline__ static void integrate(const Params&, const Voxel& v, int, float, float, float nl2,
                                                     float* I, float* T)
    {
        segments<W>(v.S, v.chi, nl2, I, T);
    }
};

// kMinCtas: CTAs per SM the register budget is sized for (1: the compiler's
// choice, 97 registers at W = 8; 1024 / NT: 64 registers, four 256-thread CTAs
// of residency, with some spilling).
// NT threads per CTA = probes per work item (a 16 x (NT / 16) part of a block,
// warps on 8 x 4 tiles as in k_solve_hdda_t); a CTA claims `chunk` consecutive
// items per queue increment.  kInfo: the block table is staged as one word per
// block (offset * 8 + state); otherwise the packed 3-bit state words.  Every
// probe accumulates J over all directions in its thread, in the order of the
// single-grid solve, so results do not depend on these choices.
// kPair (W = 8): a work unit is a pair of batches (pair_batches) walked once on
// the smaller of their two levels, 16 wavelengths per thread, or a lone batch
// (pair_lone_batch) walked alone, as dex_formal_solve_hdda's paired walk.
template <int W, int NT, bool kInfo, int kMinCtas, bool kPair = false>
__global__ void __launch_bounds__(NT, kMinCtas) k_batch_solve(const BatchParams P)
{
    extern __shared__ unsigned long long s_dyn[];
    __shared__ float s_J[kPair ? 2 * W : W][NT];
    __shared__ float s_dx[DEX_MAX_DIRS], s_dz[DEX_MAX_DIRS], s_w[DEX_MAX_DIRS];
    __shared__ unsigned int s_item;
    constexpr int kParts = 256 / NT;
    int* s_info = reinterpret_cast<int*>(s_dyn);
    const int tid = threadIdx.x;
    int cur_atm = -1, cur_batch = -1;
    unsigned int nseg_unused = 0;
    bool capped = false;
    if (P.start_ns != nullptr && tid == 0) atomicMin(P.start_ns, global_ns());

    for (;;) {
        __syncthreads();  // every thread is done with the previous claim
        if (tid == 0) s_item = atomicAdd(P.queue, (unsigned int)P.chunk);
        __syncthreads();
        const unsigned int first = s_item;
        if ((long long)first >= P.n_items) break;
        for (int c = 0; c < P.chunk; ++c) {
            const long long item = (long long)first + c;
            if (item >= P.n_items) break;
            int a = 0;
            while (a + 1 < P.n_atm && item >= P.atm[a + 1].item_base) ++a;
            const AtmDesc& A = P.atm[a];
            const long long local = item - A.item_base;
            const long long unit = local / kParts;
            const int part = (int)(local % kParts);
            const int b = (int)(unit / A.cap_active), r = (int)(unit % A.cap_active);
            if (r >= *A.n_active) continue;
            // kPair: b numbers the atmosphere's pairs, then its lone batches
            int b1 = b, b2 = -1;
            if constexpr (kPair) {
                const int n_batch = (A.n_lambda + W - 1) / W, np = pair_count(n_batch, P.pair_group);
                if (b < np) pair_batches(b, n_batch, P.pair_group, b1, b2);
                else b1 = pair_lone_batch(b - np, n_batch, P.pair_group);
            }
            __syncthreads();  // every thread is done with the previous item's shared data
            if (a != cur_atm || b != cur_batch) {
                if constexpr (kPair) {
                    // one word per block, offset * 8 + the smaller of the pair's states
                    const int nb = A.nbx * A.nbz;
                    const unsigned long long* w1 = A.words + (size_t)b1 * A.n_words;
                    const unsigned long long* w2 = A.words + (size_t)(b2 >= 0 ? b2 : b1) * A.n_words;
                    for (int q = tid; q < nb; q += NT)
                        s_info[q] = pack_block_info(A.block_offset[q], min(block_state(w1, q), block_state(w2, q)));
                } else if constexpr (kInfo) {
                    const int nb = A.nbx * A.nbz;
                    const unsigned long long* wb = A.words + (size_t)b * A.n_words;
                    for (int q = tid; q < nb; q += NT) s_info[q] = pack_block_info(A.block_offset[q], block_state(wb, q));
                } else {
                    for (int q = tid; q < A.n_words; q += NT) s_dyn[q] = A.words[(size_t)b * A.n_words + q];
                }
                if (a != cur_atm)
                    for (int q = tid; q < A.n_dir; q += NT) {
                        s_dx[q] = A.dirs[2 * q];
                        s_dz[q] = A.dirs[2 * q + 1];
                        s_w[q] = A.weights[q];
                    }
                cur_atm = a;
                cur_batch = b;
            }
#pragma unroll
            for (int w = 0; w < (kPair ? 2 * W : W); ++w) s_J[w][tid] = 0.0f;
            __syncthreads();

            const int blk0 = A.active[r];
            const int bx0 = blk0 % A.nbx, bz0 = blk0 / A.nbx;
            const int wrp = tid >> 5;
            const int i = bx0 * DEX_BLOCK + (wrp & 1) * 8 + (tid & 7);
            const int j = bz0 * DEX_BLOCK + part * (DEX_BLOCK / kParts) + (wrp >> 1) * 4 + ((tid & 31) >> 3);
            const int state0 = (kInfo || kPair ? (s_info[blk0] & 7) : block_state(s_dyn, blk0)) - 1;
            if (state0 < 0) {
                capped = true;
                continue;
            }
            Geo G;
            G.nx = A.nx;
            G.nz = A.nz;
            G.nbx = A.nbx;
            G.nbz = A.nbz;
            G.chain = A.chain;
            G.cap_active = A.cap_active;
            const size_t batch_floats = (size_t)A.cap_active * A.chain * (2 * W);
            G.batch_base = A.bricks + (size_t)b1 * batch_floats;
            set_box_full(G);
#pragma unroll
            for (int q = 0; q < 4; ++q) G.band[q] = A.band[q];
            const int mip0 = min(state0, distance_cap(G, 0.0f));
            typename StaticRec<W>::Params M{};
            for (int k = 0; k < A.n_dir; ++k) {
                const float wk = s_w[k];
                if (kPair && b2 >= 0) {
                    // the pair: 16 wavelengths along one walk
                    using PM = PairRecModel<kStoreF32, kMinCtas>;
                    const typename PM::Params M2{(long long)(b2 - b1) * (long long)batch_floats};
                    float I[2 * W], T[2 * W];
#pragma unroll
                    for (int w = 0; w < 2 * W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
                    trace_ray<2 * W, false, PM>(G, M2, b1, i, j, bx0, bz0, r, mip0, s_dx[k], s_dz[k],
                                                InfoLookup{s_info}, I, T, nseg_unused, capped);
#pragma unroll
                    for (int w = 0; w < 2 * W; ++w) s_J[w][tid] = fmaf(wk, fmaf(T[w], A.i_bc, I[w]), s_J[w][tid]);
                } else {
                    float I[W], T[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
                    if constexpr (kInfo || kPair)
                        trace_ray<W, false, StaticRec<W>>(G, M, b1, i, j, bx0, bz0, r, mip0, s_dx[k], s_dz[k],
                                                           InfoLookup{s_info}, I, T, nseg_unused, capped);
                    else
                        trace_ray<W, false, StaticRec<W>>(G, M, b1, i, j, bx0, bz0, r, mip0, s_dx[k], s_dz[k],
                                                           WordLookup{s_dyn, A.block_offset}, I, T, nseg_unused,
                                                           capped);
#pragma unroll
                    for (int w = 0; w < W; ++w) s_J[w][tid] = fmaf(wk, fmaf(T[w], A.i_bc, I[w]), s_J[w][tid]);
                }
            }
            const long long n_cells = (long long)A.nx * A.nz;
#pragma unroll
            for (int w = 0; w < (kPair ? 2 * W : W); ++w) {
                const int l = w < W ? b1 * W + w : b2 * W + (w - W);
                if ((w < W || b2 >= 0) && l < A.n_lambda) A.J[(size_t)l * n_cells + (size_t)j * A.nx + i] = s_J[w][tid];
            }
            if (P.done_ns != nullptr) {
                __syncthreads();
                if (tid == 0) atomicMax(P.done_ns + a, global_ns());
            }
        }
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
}

template <int W, int NT, bool kInfo, int kMinCtas, bool kPair = false>
cudaError_t launch_batch_t(cudaStream_t s, const BatchParams& P, int ctas, size_t smem)
{
    auto kernel = k_batch_solve<W, NT, kInfo, kMinCtas, kPair>;
    if (smem > 16 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<(unsigned)ctas, NT, smem, s>>>(P);
    return cudaSuccess;
}

template <int W, bool kOcc>
cudaError_t launch_batch_w(cudaStream_t s, const BatchParams& P, int ctas, int packet, bool info, size_t smem)
{
    switch (packet * 2 + (info ? 1 : 0)) {
        case 256 * 2: return launch_batch_t<W, 256, false, kOcc ? 4 : 1>(s, P, ctas, smem);
        case 256 * 2 + 1: return launch_batch_t<W, 256, true, kOcc ? 4 : 1>(s, P, ctas, smem);
        case 128 * 2: return launch_batch_t<W, 128, false, kOcc ? 8 : 1>(s, P, ctas, smem);
        case 128 * 2 + 1: return launch_batch_t<W, 128, true, kOcc ? 8 : 1>(s, P, ctas, smem);
        case 64 * 2: return launch_batch_t<W, 64, false, kOcc ? 16 : 1>(s, P, ctas, smem);
        case 64 * 2 + 1: return launch_batch_t<W, 64, true, kOcc ? 16 : 1>(s, P, ctas, smem);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Device address of the static scratch array on the current device.  The array's
// host-side name is not a device address, so kernels must be given this pointer.
// It is looked up on every call (a runtime table look-up, no allocation) rather
// than cached: after a cudaDeviceReset the device's context, and with it the
// array, is a new one, and a cached address would point into the old context.
cudaError_t noalloc_scratch(unsigned int** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned int*>(p);
    return cudaSuccess;
}

cudaError_t launch_batch_solve(cudaStream_t s, const BatchParams& P, int ctas, int W, int packet, bool info,
                               bool occupancy, size_t smem_bytes)
{
    cudaError_t e = cudaMemsetAsync(P.queue, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess || P.n_items == 0) return e;
    if (occupancy && W != 8) return cudaErrorInvalidValue;
    if (P.paired) {
        // pairs of batches (W = 8): one word per block staged, the compiler's budget
        // bounded at 128 registers (two 256-thread CTAs per SM)
        if (W != 8) return cudaErrorInvalidValue;
        switch (packet) {
            case 256: e = launch_batch_t<8, 256, true, 2, true>(s, P, ctas, smem_bytes); break;
            case 128: e = launch_batch_t<8, 128, true, 4, true>(s, P, ctas, smem_bytes); break;
            case 64: e = launch_batch_t<8, 64, true, 8, true>(s, P, ctas, smem_bytes); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    switch (W) {
        case 1: e = launch_batch_w<1, false>(s, P, ctas, packet, info, smem_bytes); break;
        case 2: e = launch_batch_w<2, false>(s, P, ctas, packet, info, smem_bytes); break;
        case 4: e = launch_batch_w<4, false>(s, P, ctas, packet, info, smem_bytes); break;
        case 8:
            e = occupancy ? launch_batch_w<8, true>(s, P, ctas, packet, info, smem_bytes)
                          : launch_batch_w<8, false>(s, P, ctas, packet, info, smem_bytes);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dex
