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
#include "dex_internal.h"

namespace dex {

namespace {

__host__ __device__ constexpr int level_offset(int m) { return 341 - (341 >> (2 * m)); }

__device__ __forceinline__ int block_state(const unsigned long long* words, int blk)
{
    const int wi = blk / DEX_STATES_PER_WORD, sh = DEX_STATE_BITS * (blk - wi * DEX_STATES_PER_WORD);
    return (int)((words[wi] >> sh) & 7ull);
}

template <int W>
__global__ void __launch_bounds__(256) k_solve_hdda(const HddaParams P)
{
    extern __shared__ unsigned long long s_words[];
    const int a0 = blockIdx.x;
    if (a0 >= *P.n_active) return;
    const int b = blockIdx.y;
    for (int q = threadIdx.x; q < P.n_words; q += blockDim.x) s_words[q] = P.words[(size_t)b * P.n_words + q];
    __syncthreads();

    const int blk0 = P.active[a0];
    const int bx0 = blk0 % P.nbx, bz0 = blk0 / P.nbx;
    const int i = bx0 * DEX_BLOCK + (threadIdx.x & 15), j = bz0 * DEX_BLOCK + (threadIdx.x >> 4);
    const int mip0 = block_state(s_words, blk0) - 1;
    if (mip0 < 0) {  // state words do not describe this active block
        raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
        return;
    }
    const size_t rec = 2 * W;
    const float* __restrict__ batch_base = P.bricks + (size_t)b * P.cap_active * P.chain * rec;
    const int cap = 2 * (P.nx + P.nz) + 64;
    const float ox = (float)i + 0.5f, oz = (float)j + 0.5f;

    float Jw[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Jw[w] = 0.0f;
    unsigned int nseg = 0;
    bool capped = false;

    for (int k = 0; k < P.quad.n_dir; ++k) {
        const float dx = P.quad.dx[k], dz = P.quad.dz[k];
        // a zero component counts as positive: its plane offsets stay positive
        // and their parameters (offset * inf) are +inf, so that axis never steps
        const bool px = !(dx < 0.0f), pz = !(dz < 0.0f);
        const int sx = px ? 1 : -1, sz = pz ? 1 : -1;
        const AxisParam ax = axis_param(dx), az = axis_param(dz);
        const float Ex = px ? (float)(P.nx - i) - 0.5f : (float)(-i) - 0.5f;
        const float Ez = pz ? (float)(P.nz - j) - 0.5f : (float)(-j) - 0.5f;
        const float t2 = fminf(Ex * ax.ih, Ez * az.ih);

        int mip = mip0;
        int vox = 1 << mip;
        int bxc = bx0, bzc = bz0;
        int ci = i & ~(vox - 1), cj = j & ~(vox - 1);
        const float* vbase = batch_base + (size_t)a0 * P.chain * rec + (size_t)level_offset(mip) * rec;
        float th_prev = 0.0f, tl_prev = 0.0f;
        float I[W], T[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }

        for (int it = 0;; ++it) {
            if (it >= cap) { capped = true; break; }
            const float Px = (float)(ci + (px ? vox : 0) - i) - 0.5f;
            const float Pz = (float)(cj + (pz ? vox : 0) - j) - 0.5f;
            const float tnx = Px * ax.ih, tnz = Pz * az.ih;
            const bool on_x = tnx <= tnz;
            float th = on_x ? tnx : tnz;
            float tl = plane_lo(on_x ? Px : Pz, on_x ? ax : az, th);
            if (th < th_prev) { th = th_prev; tl = tl_prev; }
            if (mip >= 0) {
                const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
                const int lx = (ci - bxc * DEX_BLOCK) >> mip, lz = (cj - bzc * DEX_BLOCK) >> mip;
                const Record<W> r = load_record<W>(vbase + (size_t)(lz * (DEX_BLOCK >> mip) + lx) * rec);
                const float nl2 = len * kNegLog2e;
#pragma unroll
                for (int w = 0; w < W; ++w) segment(r.S[w], r.chi[w], nl2, len, I[w], T[w]);
                nseg += (th > th_prev);
            }
            th_prev = th;
            tl_prev = tl;
            if (th >= t2) break;

            const int ci_old = ci, cj_old = cj, vox_old = vox;
            if (on_x) ci += sx * vox; else cj += sz * vox;
            if ((unsigned)ci >= (unsigned)P.nx || (unsigned)cj >= (unsigned)P.nz) { capped = true; break; }
            const int nbx_ = ci >> 4, nbz_ = cj >> 4;
            if (nbx_ == bxc && nbz_ == bzc) continue;
            // entered another block
            bxc = nbx_;
            bzc = nbz_;
            const int blk = bzc * P.nbx + bxc;
            const int mip_new = block_state(s_words, blk) - 1;
            if (mip_new != mip) {
                // MIP-0 cell entered: exact on the stepped axis, from p(t) on the other
                int m0x, m0z;
                if (on_x) {
                    m0x = px ? ci : ci + vox_old - 1;
                    const int zf = __float2int_rd(fmaf(th, dz, oz));
                    m0z = min(max(zf, cj_old), cj_old + vox_old - 1);
                } else {
                    m0z = pz ? cj : cj + vox_old - 1;
                    const int xf = __float2int_rd(fmaf(th, dx, ox));
                    m0x = min(max(xf, ci_old), ci_old + vox_old - 1);
                }
                mip = mip_new;
                vox = mip >= 0 ? (1 << mip) : DEX_BLOCK;
                ci = m0x & ~(vox - 1);
                cj = m0z & ~(vox - 1);
            }
            if (mip >= 0) {
                const int a = P.block_offset[blk];
                vbase = batch_base + (size_t)a * P.chain * rec + (size_t)level_offset(mip) * rec;
            }
        }
        const float wk = P.quad.w[k];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float Iw = fmaf(T[w], P.i_bc, I[w]);
            Jw[w] = fmaf(wk, Iw, Jw[w]);
            const int l = b * W + w;
            if (P.I != nullptr && l < P.n_lambda)
                P.I[((size_t)l * P.quad.n_dir + k) * P.n_cells + (size_t)j * P.nx + i] = Iw;
        }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int l = b * W + w;
        if (l < P.n_lambda) P.J[(size_t)l * P.n_cells + (size_t)j * P.nx + i] = Jw[w];
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    if (P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)nseg);
}

}  // namespace

cudaError_t launch_solve_hdda(cudaStream_t s, const HddaParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W) {
#define DEX_LAUNCH(WW)                                                                              \
    case WW:                                                                                        \
        if (smem > 48 * 1024)                                                                       \
            e = cudaFuncSetAttribute(k_solve_hdda<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)smem);                                                    \
        if (e == cudaSuccess) k_solve_hdda<WW><<<grid, 256, smem, s>>>(P);                          \
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
