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
// voxel on entering empty space, forcing t_h > t) with exact bookkeeping.  Every
// ray also has a step cap; exceeding it sets DEX_ERR_TRAVERSAL_CAP.
#include "hdda.cuh"

namespace dex {

namespace {

// Static voxel model: a record holds (S, chi) for the W wavelengths of a batch.
template <int W>
struct StaticModel {
    static constexpr int kStride = 2 * W;
    static constexpr bool kPerBatch = true;
    struct Params {
        int unused;
    };
    using Voxel = Record<W>;
    __device__ __forceinline__ static Voxel load(const float* p) { return load_record<W>(p); }
    __device__ __forceinline__ static void integrate(const Params&, const Voxel& v, int, float, float, float nl2,
                                                     float* I, float* T)
    {
#pragma unroll
        for (int w = 0; w < W; ++w) segment(v.S[w], v.chi[w], nl2, I[w], T[w]);
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
    const size_t smem = sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W) {
#define DEX_LAUNCH(WW)                                                                   \
    case WW:                                                                             \
        if (P.seg_count) e = launch_hdda_kernel(k_solve_hdda_t<WW, true, StaticModel<WW>>, grid, smem, s, P, typename StaticModel<WW>::Params{}); \
        else e = launch_hdda_kernel(k_solve_hdda_t<WW, false, StaticModel<WW>>, grid, smem, s, P, typename StaticModel<WW>::Params{}); \
        break;
        DEX_LAUNCH(1)
        DEX_LAUNCH(2)
        DEX_LAUNCH(4)
        DEX_LAUNCH(8)
#undef DEX_LAUNCH
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dex
