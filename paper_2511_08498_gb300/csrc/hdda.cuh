// Hierarchical DDA traversal over the sparse, mipmapped block grid, shared by
// the static solver (k_hdda.cu) and the Core-and-Voigt solver (k_cav.cu).
// See k_hdda.cu for the description of the traversal.
#pragma once

#include "dex_internal.h"

namespace dex {

__host__ __device__ constexpr int level_offset(int m) { return 341 - (341 >> (2 * m)); }

// Geometry of one sparse grid as the traversal needs it.
struct Geo {
    int nx, nz, nbx, nbz, chain, cap_active;
    int x_lo, x_hi, z_lo, z_hi;  // cell faces bounding the non-empty blocks
    const float* batch_base;     // bricks of the wavelength batch being solved
    float band[4];               // distance thresholds, padded (pad_bands)
};

// Rays end where they leave this box: beyond it every block is empty and adds
// nothing to I or T.  The whole grid, where the box is not known.
__device__ __forceinline__ void set_box_full(Geo& G)
{
    G.x_lo = 0;
    G.x_hi = G.nx;
    G.z_lo = 0;
    G.z_hi = G.nz;
}

// Highest level a block first entered at ray parameter t >= 0 may use: the
// number of thresholds band[m-1] <= t (Section 4.1: the near field at full
// resolution, coarser levels only further out).
__device__ __forceinline__ int distance_cap(const Geo& G, float t)
{
    return (G.band[0] <= t) + (G.band[1] <= t) + (G.band[2] <= t) + (G.band[3] <= t);
}

__device__ __forceinline__ int block_state(const unsigned long long* words, int blk)
{
    const int wi = blk / DEX_STATES_PER_WORD, sh = DEX_STATE_BITS * (blk - wi * DEX_STATES_PER_WORD);
    return (int)((words[wi] >> sh) & 7ull);
}

// Block lookups of the traversal: key(blk) once per block entered, then its
// state (0 = empty, level + 1) and, for non-empty blocks, its brick offset.
//
// WordLookup: the packed 3-bit states (staged in shared memory) and the global
// offset table, read only for non-empty blocks.
struct WordLookup {
    const unsigned long long* words;
    const int* offset;
    __device__ __forceinline__ int key(int blk) const { return blk; }
    __device__ __forceinline__ int state(int k) const { return block_state(words, k); }
    __device__ __forceinline__ int offset_of(int k) const { return offset[k]; }
};

// InfoLookup: one shared-memory word per block, offset * 8 + state (offset -1
// for empty blocks), so a block crossing costs one shared load.
struct InfoLookup {
    const int* info;
    __device__ __forceinline__ int key(int blk) const { return info[blk]; }
    __device__ __forceinline__ int state(int k) const { return k & 7; }
    __device__ __forceinline__ int offset_of(int k) const { return k >> 3; }
};


__device__ __forceinline__ int pack_block_info(int offset, int state) { return offset * 8 + state; }

namespace {
// A record of zeros (any static record format up to 32 floats).  Integrating it
// changes nothing: tau = 0, so 2^x = 1, 1 - e^{-tau} = 0, I += T * 0 and T *= 1.
// Rays of models with kZeroNoop read it in empty blocks instead of branching
// around the update.
__device__ __align__(32) float g_zero_record[32] = {0.0f};
}  // namespace

// Voxel models whose records are float32 brick rows (BrickFmt: a row's S
// values, then its chi values) declare kSplit = true, the floats between x
// neighbours of a row as kSplitStride, and load the record of a voxel from its
// S pointer and the distance to its chi (Model::load_split).
template <class M, class = void>
struct SplitOf {
    static constexpr bool value = false;
    static constexpr int stride = 0;
};
template <class M>
struct SplitOf<M, decltype((void)M::kSplit)> {
    static constexpr bool value = M::kSplit;
    static constexpr int stride = M::kSplitStride;
};

// Record load of a voxel model: Model::load(M, p) where the model declares it
// (its records need the launch parameters, e.g. a second batch's offset),
// Model::load(p) otherwise.
template <class Model>
__device__ __forceinline__ auto model_load(const typename Model::Params& M, const float* p)
    -> decltype(Model::load(M, p))
{
    return Model::load(M, p);
}
template <class Model>
__device__ __forceinline__ auto model_load(const typename Model::Params&, const float* p) -> decltype(Model::load(p))
{
    return Model::load(p);
}

// Two batches' records of one voxel, `off` floats apart, in format ST: the
// wavelengths of the first are 0..7 of the walk, those of the second 8..15 (a
// walk shared by a pair of batches on their common levels).  Empty blocks are
// stepped over without a record (the zero record has no second batch beside it).
template <int ST, int MINB>
struct PairRecModel {
    static constexpr int kStride = RecFmt<8, ST>::kStride;
    static constexpr bool kSplit = BrickFmt<8, ST>::kSplit;
    static constexpr int kSplitStride = BrickFmt<8, ST>::kX;
    static constexpr bool kPerBatch = true;
    static constexpr int kMinBlocks = MINB;
    static constexpr bool kEarlyLoad = ST == kStoreF32;
    static constexpr bool kZeroNoop = false;
    struct Params {
        long long off;
    };
    struct Voxel {
        Record<8> a, b;
    };
    __device__ __forceinline__ static Voxel load(const Params& M, const float* p)
    {
        Voxel v;
        v.a = RecFmt<8, ST>::load(p);
        v.b = RecFmt<8, ST>::load(p + M.off);
        return v;
    }
    __device__ __forceinline__ static Voxel load_split(const Params& M, const float* p, int coff)
    {
        Voxel v;
        v.a = BrickFmt<8, ST>::load(p, coff);
        v.b = BrickFmt<8, ST>::load(p + M.off, coff);
        return v;
    }
    __device__ __forceinline__ static void integrate(const Params&, const Voxel& v, int, float, float, float nl2,
                                                     float* I, float* T)
    {
        segments<8>(v.a.S, v.a.chi, nl2, I, T);
        segments<8>(v.b.S, v.b.chi, nl2, I + 8, T + 8);
    }
};

// Voxel models: Model::kStride floats per voxel record, Model::kPerBatch whether
// records differ per wavelength batch, Model::kEarlyLoad whether the record is
// loaded at the top of each step, Model::kZeroNoop whether a record of zeros
// integrates to no change, Model::Voxel / load / integrate the per-segment
// update of the W wavelengths of batch b along propagation (wx, wz).
//
// One ray from the centre of cell (i, j) (in active block a0 = (bx0, bz0), whose
// level is mip0) along d = (dx, dz): accumulates I and T (initialised by the
// caller) over the traversal; L looks up the batch's block states and offsets.
// EXT: the emission of the probe's own voxel (the first segment) is left out.
//
// Each step integrates the voxel it leaves and steps to the next voxel of the
// same level; only a step that leaves the block (one divergent branch) looks up
// the next block: after the integration for models with kZeroNoop (the
// transmission test then sees the block's last segment), before it otherwise.  A ray's block indices change monotonically and it takes at
// most 2 * 16 steps in a block, so the grid bounds check also bounds the loop.
template <int W, bool COUNT, class Model, class Lookup, bool EXT = false>
__device__ __forceinline__ void trace_ray(const Geo& G, const typename Model::Params& M, int b, int i, int j,
                                          int bx0, int bz0, int a0, int mip0, float dx, float dz,
                                          const Lookup& L, float* I, float* T, unsigned int& nseg, bool& capped)
{
    constexpr int REC = Model::kStride;
    constexpr bool kZero = Model::kZeroNoop;
    constexpr bool kSplit = SplitOf<Model>::value;
    constexpr int XS = kSplit ? SplitOf<Model>::stride : REC;  // floats between x neighbours of a row
    static_assert(!kSplit || Model::kEarlyLoad, "float32 brick rows are read at the top of the step");
    const float* __restrict__ batch_base = G.batch_base;
    const float ox = (float)i + 0.5f, oz = (float)j + 0.5f;
    const bool negx = dx < 0.0f, negz = dz < 0.0f;
    const int sx = negx ? -1 : 1, sz = negz ? -1 : 1;
    const AxisParam ax = axis_param(dx), az = axis_param(dz);
    // exit plane offsets: the faces of the box around the non-empty blocks
    const float Ex = (float)((negx ? G.x_lo : G.x_hi) - i) - 0.5f;
    const float Ez = (float)((negz ? G.z_lo : G.z_hi) - j) - 0.5f;
    const float t2 = fminf(Ex * ax.ih, Ez * az.ih);

    // tracer state: level, voxel size, block, block-local voxel, far-face plane offsets
    int mip = mip0, vox = 1 << mip0, side = DEX_BLOCK >> mip0;
    float fvox = (float)vox;
    int bxc = bx0, bzc = bz0;
    int lx = (i - bx0 * DEX_BLOCK) >> mip, lz = (j - bz0 * DEX_BLOCK) >> mip;
    float Px = (float)(bx0 * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
    float Pz = (float)(bz0 * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox - j) - 0.5f;
    // record (S) of the current voxel: rows of side voxels, x neighbours XS floats apart
    const float* rp = batch_base + ((size_t)a0 * G.chain + level_offset(mip) + lz * side) * REC + lx * XS;
    float th_prev = 0.0f, tl_prev = 0.0f;
    // the step left the block: look up the next one and re-initialise the tracer
    // there (false: the ray ends)
    auto enter = [&](bool on_x, float th) -> bool {
        // early termination: once every transmission has underflowed to exactly
        // zero the rest of the ray adds exact zeros, so stopping leaves I and T
        // bit-identical
        if (all_opaque<W>(T)) return false;
        if (on_x) bxc += sx;
        else bzc += sz;
        if ((unsigned)bxc >= (unsigned)G.nbx || (unsigned)bzc >= (unsigned)G.nbz) {
            capped = true;
            return false;
        }
        const int key = L.key(bzc * G.nbx + bxc);
        const int st = L.state(key) - 1;
        const int mip_new = st < 0 ? -1 : min(st, distance_cap(G, th));
        if (mip_new == mip) {
            if (on_x) lx = negx ? side - 1 : 0;
            else lz = negz ? side - 1 : 0;
        } else {
            // MIP-0 cell entered: exact on the stepped axis, from p(t) on the
            // other one, clamped to the voxel just left (the block index on that
            // axis is unchanged)
            const int vox_old = vox;
            int m0x, m0z;
            if (on_x) {
                m0x = bxc * DEX_BLOCK + (negx ? DEX_BLOCK - 1 : 0);
                const int lo = bzc * DEX_BLOCK + lz * vox_old;
                m0z = min(max(__float2int_rd(fmaf(th, dz, oz)), lo), lo + vox_old - 1);
            } else {
                m0z = bzc * DEX_BLOCK + (negz ? DEX_BLOCK - 1 : 0);
                const int lo = bxc * DEX_BLOCK + lx * vox_old;
                m0x = min(max(__float2int_rd(fmaf(th, dx, ox)), lo), lo + vox_old - 1);
            }
            mip = mip_new;
            const int shift = mip >= 0 ? mip : 4;
            vox = 1 << shift;
            fvox = (float)vox;
            side = DEX_BLOCK >> shift;
            lx = (m0x - bxc * DEX_BLOCK) >> shift;
            lz = (m0z - bzc * DEX_BLOCK) >> shift;
            Px = (float)(bxc * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
            Pz = (float)(bzc * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox - j) - 0.5f;
        }
        if (mip >= 0)
            rp = batch_base + ((size_t)L.offset_of(key) * G.chain + level_offset(mip) + lz * side) * REC + lx * XS;
        else if (kZero)
            rp = g_zero_record;
        return true;
    };
    typename Model::Voxel cur;

    // unrolled four times (twice and eight times measured slower on the 1024^2
    // benchmark solve, for the single- and the two-batch model)
#pragma unroll 4
    for (int it = 0;; ++it) {
        // models with kEarlyLoad issue the current voxel's record before the
        // stepping and crossing bookkeeping, which then hides its latency
        if constexpr (Model::kEarlyLoad) {
            if (kZero || mip >= 0) {
                if constexpr (kSplit) cur = Model::load_split(M, rp, side * XS);
                else cur = model_load<Model>(M, rp);
            }
        }
        const float tnx = Px * ax.ih, tnz = Pz * az.ih;
        const bool on_x = tnx <= tnz;
        const float th = on_x ? tnx : tnz;
        const float tl = plane_lo(on_x ? Px : Pz, on_x ? ax : az, th);
        const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
        const bool last = th >= t2;
        const int cur_mip = mip;
        const float* cur_rp = rp;
        // step to the next voxel of this level (not used once last)
        bool cross;
        if (on_x) {
            lx += sx;
            Px += negx ? -fvox : fvox;
            rp += negx ? -XS : XS;
            cross = (unsigned)lx >= (unsigned)side;
        } else {
            lz += sz;
            Pz += negz ? -fvox : fvox;
            rp += negz ? -side * REC : side * REC;
            cross = (unsigned)lz >= (unsigned)side;
        }
        if constexpr (!kZero) {
            // models without a zero record enter the next block before integrating
            // (measured 2-4% faster for them on a 1024 x 512 moving medium)
            if (cross && !last && !enter(on_x, th)) break;
        }
        // integrate the voxel left (in empty blocks: the zero record, or nothing)
        if (kZero || cur_mip >= 0) {
            if constexpr (!Model::kEarlyLoad) cur = model_load<Model>(M, cur_rp);
            Model::integrate(M, cur, b, -dx, -dz, len * kNegLog2e, I, T);
            if constexpr (EXT) {
                if (it == 0) {
#pragma unroll
                    for (int w = 0; w < W; ++w) I[w] = 0.0f;
                }
            }
            if (COUNT) nseg += (cur_mip >= 0) & (th > th_prev);
        }
        if (last) break;
        th_prev = th;
        tl_prev = tl;
        if constexpr (kZero) {
            if (cross && !enter(on_x, th)) break;
        }
    }
}

// kInfo: the CTA stages one word per block (offset * 8 + state, InfoLookup;
// dynamic shared memory 4 * nbx * nbz bytes, grids of at most kInfoMaxBlocks
// blocks); otherwise the packed state words (WordLookup; 8 * n_words bytes).
template <int W, bool COUNT, class Model, bool kInfo = false, bool EXT = false>
__global__ void __launch_bounds__(256, Model::kMinBlocks) k_solve_hdda_t(const HddaParams P, const typename Model::Params M)
{
    extern __shared__ unsigned long long s_dyn[];
    __shared__ float s_J[W][256];
    const int a0 = blockIdx.x;
    if (a0 >= *P.n_active) return;
    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const unsigned long long* words_b = P.words + (size_t)b * P.n_words;
    int* s_info = reinterpret_cast<int*>(s_dyn);
    if constexpr (kInfo) {
        const int n_blocks = P.nbx * P.nbz;
        for (int q = tid; q < n_blocks; q += blockDim.x) s_info[q] = pack_block_info(P.block_offset[q], block_state(words_b, q));
    } else {
        for (int q = tid; q < P.n_words; q += blockDim.x) s_dyn[q] = words_b[q];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) s_J[w][tid] = 0.0f;
    // box around the non-empty (active) blocks, in block units
    __shared__ int s_box[4];
    if (tid < 4) s_box[tid] = (tid & 1) ? -1 : 0x7fffffff;
    __syncthreads();
    {
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
    // warp w covers an 8 x 4 tile of the block (lanes along x, then z): a warp's rays
    // meet x faces in at most 8 different iterations (16 with whole 16-cell rows),
    // while its record loads stay within the block's brick
    const int wrp = tid >> 5;
    const int i = bx0 * DEX_BLOCK + (wrp & 1) * 8 + (tid & 7);
    const int j = bz0 * DEX_BLOCK + (wrp >> 1) * 4 + ((tid & 31) >> 3);
    const int state0 = (kInfo ? (s_info[blk0] & 7) : block_state(s_dyn, blk0)) - 1;
    if (state0 < 0) {  // state words do not describe this active block
        raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
        return;
    }
    Geo G;
    G.nx = P.nx;
    G.nz = P.nz;
    G.nbx = P.nbx;
    G.nbz = P.nbz;
    G.chain = P.chain;
    G.cap_active = P.cap_active;
    G.batch_base = P.bricks + (Model::kPerBatch ? (size_t)b * P.cap_active * P.chain * Model::kStride : (size_t)0);
    G.x_lo = s_box[0] * DEX_BLOCK;
    G.x_hi = (s_box[1] + 1) * DEX_BLOCK;
    G.z_lo = s_box[2] * DEX_BLOCK;
    G.z_hi = (s_box[3] + 1) * DEX_BLOCK;
#pragma unroll
    for (int q = 0; q < 4; ++q) G.band[q] = P.band[q];
    const int mip0 = min(state0, distance_cap(G, 0.0f));
    unsigned int nseg = 0;
    bool capped = false;

    for (int k = 0; k < P.quad.n_dir; ++k) {
        const float dx = P.quad.dx[k], dz = P.quad.dz[k];
        float I[W], T[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
        if constexpr (kInfo)
            trace_ray<W, COUNT, Model, InfoLookup, EXT>(G, M, b, i, j, bx0, bz0, a0, mip0, dx, dz,
                                                        InfoLookup{s_info}, I, T, nseg, capped);
        else
            trace_ray<W, COUNT, Model, WordLookup, EXT>(G, M, b, i, j, bx0, bz0, a0, mip0, dx, dz,
                                                        WordLookup{s_dyn, P.block_offset}, I, T, nseg, capped);
        const float wk = P.quad.w[k];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float Iw = fmaf(T[w], P.i_bc, I[w]);
            s_J[w][tid] = fmaf(wk, Iw, s_J[w][tid]);
            const int l = b * W + w;
            if (P.I != nullptr && l < P.n_lambda)
                P.I[((size_t)l * P.quad.n_dir + k) * P.n_cells + (size_t)j * P.nx + i] = Iw;
        }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int l = b * W + w;
        if (l < P.n_lambda) P.J[(size_t)l * P.n_cells + (size_t)j * P.nx + i] = s_J[w][tid];
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)nseg);
}


}  // namespace dex
