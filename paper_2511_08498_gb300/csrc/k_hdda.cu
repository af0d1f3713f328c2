// Hierarchical DDA formal solver over the sparse, mipmapped block grid
// (Section 2.3, Algorithm 1, with the robustness requirements of Section 2.3.1).
//
// One CTA per (active block, wavelength batch); one thread per probe cell of
// the block, walking every quadrature direction (J accumulates in registers).
// The packed 3-bit block states of the batch are staged in shared memory: they
// are the structure the traversal consults at every block crossing.
//
// Traversal of one ray p(t) = p_c + t d:
//  * inside a region of constant voxel size vox = 2^mip (16 for an empty block,
//    mip = -1) it is the DDA of Amanatides & Woo: the next plane on each axis is
//    at the voxel's far face, the nearer one ends the segment;
//  * segments in non-empty blocks are integrated with the voxel's (S, chi) record
//    at level mip; empty blocks are crossed in one step and add nothing;
//  * on entering a block with another level the tracer is re-initialised: the
//    MIP-0 cell entered is known exactly on the stepped axis (the plane just
//    crossed) and taken from p(t) on the other axis, clamped to the voxel the ray
//    was in; both are floored to the new voxel size.
// Plane parameters are two-float sums (see AxisParam) and t never decreases: a
// plane found behind the ray (rounding after a re-initialisation) yields a
// zero-length step.  These replace the paper's two nudges (advancing t by 1e-2
// voxel on entering empty space, forcing t_h > t) with exact bookkeeping.  A ray
// ends where it leaves the box around the non-empty blocks (nothing beyond it
// adds to I or T); a ray that would step out of the grid before that sets
// DEX_ERR_TRAVERSAL_CAP.
#include "hdda.cuh"

namespace dex {

namespace {

// Static voxel model: a record holds (S, chi) for the W wavelengths of a batch,
// stored in format ST (float32, bfloat16 or scaled float16; see RecFmt).
template <int W, int ST = kStoreF32>
struct StaticModel {
    static constexpr int kStride = RecFmt<W, ST>::kStride;
    static constexpr bool kSplit = BrickFmt<W, ST>::kSplit;  // float32: brick rows of S, then chi
    static constexpr int kSplitStride = BrickFmt<W, ST>::kX;
    static constexpr bool kPerBatch = true;
    static constexpr int kMinBlocks = 4;  // CTAs per SM the register budget targets
    // record loaded at the top of each step: -3.3% (float32) on the 1024^2 benchmark
    // solve; +5% with the bfloat16 / float16 unpacking (register pressure)
    static constexpr bool kEarlyLoad = ST == kStoreF32;
    static constexpr bool kZeroNoop = true;  // zero records integrate to no change
    struct Params {
        int unused;
    };
    using Voxel = Record<W>;
    __device__ __forceinline__ static Voxel load(const float* p) { return RecFmt<W, ST>::load(p); }
    __device__ __forceinline__ static Voxel load_split(const Params&, const float* p, int coff)
    {
        return BrickFmt<W, ST>::load(p, coff);
    }
    __device__ __forceinline__ static void integrate(const Params&, const Voxel& v, int, float, float, float nl2,
                                                     float* I, float* T)
    {
        segments<W>(v.S, v.chi, nl2, I, T);
    }
};

template <typename K, typename MP>
cudaError_t launch_hdda_kernel(K kernel, dim3 grid, size_t smem, cudaStream_t s, const HddaParams& P, const MP& M)
{
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 256, smem, s>>>(P, M);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_solve_hdda(cudaStream_t s, const HddaParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    if (P.traversal == DEX_TRAVERSAL_PAIRED) {
        if (!solve_hdda_paired_applies(P)) return cudaErrorNotSupported;
        return launch_solve_hdda_paired(s, P);
    }
    if (solve_hdda_shared_applies(P)) return launch_solve_hdda_shared(s, P);
    if (P.exclude_own) {
        // own-voxel emission left out: W = 8, float32 records (the MALI path)
        if (P.W != 8 || P.storage != kStoreF32) return cudaErrorNotSupported;
        const long long nb = (long long)P.nbx * P.nbz;
        const bool inf = nb <= kInfoMaxBlocks;
        const size_t sm = inf ? sizeof(int) * (size_t)nb : sizeof(unsigned long long) * (size_t)P.n_words;
        dim3 g((unsigned)P.cap_active, (unsigned)P.n_batch);
        using SM8 = StaticModel<8, kStoreF32>;
        cudaError_t e;
        if (inf && P.seg_count) e = launch_hdda_kernel(k_solve_hdda_t<8, true, SM8, true, true>, g, sm, s, P, SM8::Params{});
        else if (inf) e = launch_hdda_kernel(k_solve_hdda_t<8, false, SM8, true, true>, g, sm, s, P, SM8::Params{});
        else if (P.seg_count) e = launch_hdda_kernel(k_solve_hdda_t<8, true, SM8, false, true>, g, sm, s, P, SM8::Params{});
        else e = launch_hdda_kernel(k_solve_hdda_t<8, false, SM8, false, true>, g, sm, s, P, SM8::Params{});
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    // W = 8 on grids of at most kInfoMaxBlocks blocks: one shared-memory word per
    // block (InfoLookup); otherwise the packed state words (WordLookup)
    const long long n_blocks = (long long)P.nbx * P.nbz;
    const bool info = P.W == 8 && n_blocks <= kInfoMaxBlocks;
    const size_t smem = info ? sizeof(int) * (size_t)n_blocks : sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W * 4 + P.storage) {
#define MP_(WW, ST) typename StaticModel<WW, ST>::Params{}
#define DEX_LAUNCH(WW, ST)                                                                                   \
    case WW * 4 + ST:                                                                                        \
        if (P.seg_count)                                                                                     \
            e = launch_hdda_kernel(k_solve_hdda_t<WW, true, StaticModel<WW, ST>>, grid, smem, s, P, MP_(WW, ST));   \
        else                                                                                                 \
            e = launch_hdda_kernel(k_solve_hdda_t<WW, false, StaticModel<WW, ST>>, grid, smem, s, P, MP_(WW, ST));  \
        break;
#define DEX_LAUNCH_INFO(ST)                                                                                  \
    case 8 * 4 + ST:                                                                                         \
        if (info && P.seg_count)                                                                             \
            e = launch_hdda_kernel(k_solve_hdda_t<8, true, StaticModel<8, ST>, true>, grid, smem, s, P, MP_(8, ST));  \
        else if (info)                                                                                       \
            e = launch_hdda_kernel(k_solve_hdda_t<8, false, StaticModel<8, ST>, true>, grid, smem, s, P, MP_(8, ST)); \
        else if (P.seg_count)                                                                                \
            e = launch_hdda_kernel(k_solve_hdda_t<8, true, StaticModel<8, ST>>, grid, smem, s, P, MP_(8, ST));     \
        else                                                                                                 \
            e = launch_hdda_kernel(k_solve_hdda_t<8, false, StaticModel<8, ST>>, grid, smem, s, P, MP_(8, ST));    \
        break;
        DEX_LAUNCH(1, kStoreF32)
        DEX_LAUNCH(2, kStoreF32)
        DEX_LAUNCH(4, kStoreF32)
        DEX_LAUNCH_INFO(kStoreF32)
        DEX_LAUNCH(4, kStoreBF16)
        DEX_LAUNCH_INFO(kStoreBF16)
        DEX_LAUNCH(4, kStoreF16)
        DEX_LAUNCH_INFO(kStoreF16)
#undef DEX_LAUNCH_INFO
#undef DEX_LAUNCH
#undef MP_
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dex

namespace dex {

int record_floats(int W, int storage)
{
    if (storage == kStoreF32) return 2 * W;
    if (storage == kStoreBF16) return W;
    if (storage == kStoreF16) return 4 + W;
    return 0;
}

}  // namespace dex
