// Radiance cascades around the hierarchical DDA (the formal solution of the
// paper's code, Section 4.1 "Model Configuration"): cascade i has probes on a
// lattice of spacing 2^i, n0 4^i directions and the radiance interval
// [t0 4^(i-1), t0 4^i] (cascade 0: [0, t0]); its intervals are traced through the
// sparse mipmapped grid at min(block level, the cascade's level cap).
//
// One launch per cascade, from the top down, fuses the trace with the merge:
//   L = I + T R,  R = i_bc where the ray left the grid inside its interval (and
//   on the top cascade), else the bilinear interpolation at this probe of the
//   mean over the 4 child directions (4k .. 4k+3) of the cascade above (its 4
//   nearest probes, indices clamped at the lattice edge).
// Thread = (direction, probe) of one wavelength batch.  On the lower cascades
// probes run fastest, so the lanes of a warp trace parallel rays from
// neighbouring probes; on the upper ones (long intervals from probes 16 or more
// cells apart) directions run fastest, so a warp's rays fan out from one probe
// and read neighbouring bricks.  Cascade 0 skips
// probes in empty blocks (J is not defined there).  A final kernel averages the
// cascade-0 radiance over its directions into J.
//
// The tracer starts at t_s: the entry cell is floor(p(t_s)) (a rounding that
// lands in the next cell back only yields a zero-length first step), plane
// offsets from the probe are exact (probes sit at multiples of 1/2), and the
// last segment is clipped at min(t_e, grid exit).
#include "dex_internal.h"

namespace dex {

namespace {

__host__ __device__ constexpr int rc_level_offset(int m) { return 341 - (341 >> (2 * m)); }

__device__ __forceinline__ int rc_block_state(const unsigned long long* words, int blk)
{
    const int wi = blk / DEX_STATES_PER_WORD, sh = DEX_STATE_BITS * (blk - wi * DEX_STATES_PER_WORD);
    return (int)((words[wi] >> sh) & 7ull);
}

// Block state of the walk: NB = 1 the batch's own, NB = 2 the smaller of the
// two batches' states (0 = empty wins).
template <int NB>
__device__ __forceinline__ int rc_walk_state(const unsigned long long* w1, const unsigned long long* w2, int blk)
{
    const int s1 = rc_block_state(w1, blk);
    return NB == 2 ? min(s1, rc_block_state(w2, blk)) : s1;
}

// Emission I and transmission T of the interval [t_s, t_e] of the ray o + t d
// through the sparse mipmapped grid; returns true when the ray leaves the grid
// before t_e.  NB = 2: two wavelength batches (bricks `off` floats apart, state
// words words2) along one walk on the smaller of their levels; I and T hold
// 2 W values, the second batch's from index W.
template <int W, bool COUNT, int ST, int NB = 1>
__device__ __forceinline__ bool rc_interval(const RcParams& P, const float* __restrict__ base, long long off,
                                            const unsigned long long* __restrict__ words,
                                            const unsigned long long* __restrict__ words2, float ox, float oz,
                                            float dx, float dz, float* I, float* T, unsigned int& nseg,
                                            bool& capped)
{
    using BF = BrickFmt<W, ST>;
    constexpr int REC = BF::kRec;
    const bool negx = dx < 0.0f, negz = dz < 0.0f;
    const int sx = negx ? -1 : 1, sz = negz ? -1 : 1;
    const AxisParam ax = axis_param(dx), az = axis_param(dz);
    const float t_exit = fminf((negx ? -ox : (float)P.nx - ox) * ax.ih, (negz ? -oz : (float)P.nz - oz) * az.ih);
    const bool left = t_exit <= P.t_e;
    const float t_end = fminf(t_exit, P.t_e);
    if (!(t_end > P.t_s)) return true;
    const int cap = 2 * (P.nx + P.nz) + 64;

    // entry cell, block, level and voxel at t_s
    const int cx = min(max(__float2int_rd(fmaf(P.t_s, dx, ox)), 0), P.nx - 1);
    const int cz = min(max(__float2int_rd(fmaf(P.t_s, dz, oz)), 0), P.nz - 1);
    int bxc = cx >> 4, bzc = cz >> 4;
    int blk = bzc * P.nbx + bxc;
    int st = rc_walk_state<NB>(words, words2, blk) - 1;
    int mip = st < 0 ? -1 : min(st, P.level_cap);
    int shift = mip >= 0 ? mip : 4;
    int vox = 1 << shift, side = DEX_BLOCK >> shift;
    int lx = (cx - bxc * DEX_BLOCK) >> shift, lz = (cz - bzc * DEX_BLOCK) >> shift;
    float Px = (float)(bxc * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox) - ox;
    float Pz = (float)(bzc * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox) - oz;
    const float* rp = base;
    if (mip >= 0)
        rp = base + BF::offset((long long)P.block_offset[blk] * P.chain + rc_level_offset(mip), lz, lx, side);
    float th_prev = P.t_s, tl_prev = 0.0f;

    Record<W> r, r2;
    for (int it = 0;; ++it) {
        // the current voxel's record is issued first: the stepping and crossing
        // bookkeeping below hides its latency
        if (mip >= 0) {
            r = BF::load(rp, BF::chi_off(side));
            if constexpr (NB == 2) r2 = BF::load(rp + off, BF::chi_off(side));
        }
        const float tnx = Px * ax.ih, tnz = Pz * az.ih;
        const bool on_x = tnx <= tnz;
        float th = on_x ? tnx : tnz;
        float tl = plane_lo(on_x ? Px : Pz, on_x ? ax : az, th);
        const bool last = th >= t_end;
        if (last) {  // clipped at the interval end (or the grid exit)
            th = t_end;
            tl = 0.0f;
        }
        const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
        const int cur_mip = mip;
        if (!last) {
            if (it >= cap) { capped = true; break; }
            const float fv = (float)vox;
            bool cross;
            if (on_x) {
                lx += sx;
                Px += negx ? -fv : fv;
                rp += negx ? -BF::kX : BF::kX;
                cross = (unsigned)lx >= (unsigned)side;
            } else {
                lz += sz;
                Pz += negz ? -fv : fv;
                rp += negz ? -side * REC : side * REC;
                cross = (unsigned)lz >= (unsigned)side;
            }
            if (cross && all_opaque<NB * W>(T)) break;  // the rest adds exact zeros
            if (cross) {
                const int bxn = bxc + (on_x ? sx : 0), bzn = bzc + (on_x ? 0 : sz);
                if ((unsigned)bxn >= (unsigned)P.nbx || (unsigned)bzn >= (unsigned)P.nbz) {
                    capped = true;
                    break;
                }
                blk = bzn * P.nbx + bxn;
                st = rc_walk_state<NB>(words, words2, blk) - 1;
                const int mip_new = st < 0 ? -1 : min(st, P.level_cap);
                if (mip_new == mip) {
                    if (on_x) lx = negx ? side - 1 : 0;
                    else lz = negz ? side - 1 : 0;
                } else {
                    // MIP-0 cell entered: exact on the stepped axis, from p(t) on the
                    // other one, clamped to the voxel just left
                    const int vo = vox;
                    int m0x, m0z;
                    if (on_x) {
                        m0x = bxn * DEX_BLOCK + (negx ? DEX_BLOCK - 1 : 0);
                        const int lo = bzc * DEX_BLOCK + lz * vo;
                        m0z = min(max(__float2int_rd(fmaf(th, dz, oz)), lo), lo + vo - 1);
                    } else {
                        m0z = bzn * DEX_BLOCK + (negz ? DEX_BLOCK - 1 : 0);
                        const int lo = bxc * DEX_BLOCK + lx * vo;
                        m0x = min(max(__float2int_rd(fmaf(th, dx, ox)), lo), lo + vo - 1);
                    }
                    mip = mip_new;
                    shift = mip >= 0 ? mip : 4;
                    vox = 1 << shift;
                    side = DEX_BLOCK >> shift;
                    lx = (m0x - bxn * DEX_BLOCK) >> shift;
                    lz = (m0z - bzn * DEX_BLOCK) >> shift;
                    Px = (float)(bxn * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox) - ox;
                    Pz = (float)(bzn * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox) - oz;
                }
                bxc = bxn;
                bzc = bzn;
                if (mip >= 0)
                    rp = base + BF::offset((long long)P.block_offset[blk] * P.chain + rc_level_offset(mip), lz, lx, side);
            }
        }
        if (cur_mip >= 0) {
            segments<W>(r.S, r.chi, len * kNegLog2e, I, T);
            if constexpr (NB == 2) segments<W>(r2.S, r2.chi, len * kNegLog2e, I + W, T + W);
            if (COUNT) nseg += NB * (th > th_prev);
        }
        if (last) break;
        th_prev = th;
        tl_prev = tl;
    }
    return left;
}

// NB = 1: blockIdx.y is the batch (with P.paired: the lone batch
// pair_lone_batch(blockIdx.y)); NB = 2: the pair pair_batches(blockIdx.y), one
// walk for both batches on the smaller of their levels.
template <int W, bool COUNT, int ST, int NB>
__global__ void __launch_bounds__(256, NB == 1 ? 4 : 2) k_rc_cascade(const RcParams P)
{
    int b = blockIdx.y, b2 = blockIdx.y;
    if constexpr (NB == 2) pair_batches(blockIdx.y, P.n_batch, P.pair_group, b, b2);
    else if (P.paired) b = b2 = pair_lone_batch(blockIdx.y, P.n_batch, P.pair_group);
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_probe = (long long)P.pnx * P.pnz;
    if (g >= n_probe * P.n_dir) return;
    int k, p;
    if (P.dir_fastest) {  // lanes: neighbouring directions of one probe
        p = (int)(g / P.n_dir);
        k = (int)(g - (long long)p * P.n_dir);
    } else {              // lanes: neighbouring probes, one direction
        k = (int)(g / n_probe);
        p = (int)(g - (long long)k * n_probe);
    }
    const int px = p % P.pnx, pz = p / P.pnx;
    const unsigned long long* words = P.words + (size_t)b * P.n_words;
    const unsigned long long* words2 = P.words + (size_t)b2 * P.n_words;
    if (P.spacing == 1) {  // cascade 0: probes only in non-empty blocks
        if (rc_block_state(words, (pz >> 4) * P.nbx + (px >> 4)) == 0) return;
    }
    constexpr int REC = RecFmt<W, ST>::kStride;
    const size_t batch_floats = (size_t)P.cap_active * P.chain * REC;
    const float* base = P.bricks + (size_t)b * batch_floats;
    const long long off = (long long)(b2 - b) * (long long)batch_floats;
    const float ox = (float)P.spacing * ((float)px + 0.5f), oz = (float)P.spacing * ((float)pz + 0.5f);
    const float dx = P.dirs[2 * k], dz = P.dirs[2 * k + 1];
    float I[NB * W], T[NB * W];
#pragma unroll
    for (int w = 0; w < NB * W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
    unsigned int nseg = 0;
    bool capped = false;
    const bool left = rc_interval<W, COUNT, ST, NB>(P, base, off, words, words2, ox, oz, dx, dz, I, T, nseg, capped);

#pragma unroll
    for (int q = 0; q < NB; ++q) {
    const int bq = q == 0 ? b : b2;
    float R[W];
#pragma unroll
    for (int w = 0; w < W; ++w) R[w] = P.i_bc;
    if (!left && P.upper != nullptr) {
        // bilinear stencil on the coarser lattice: this probe sits at (p + 1/2)/2 - 1/2
        const int qnx = P.pnx >> 1, qnz = P.pnz >> 1;
        const float ux = 0.5f * ((float)px + 0.5f) - 0.5f, uz = 0.5f * ((float)pz + 0.5f) - 0.5f;
        const int x0 = (int)floorf(ux), z0 = (int)floorf(uz);
        const float fx = ux - (float)x0, fz = uz - (float)z0;
        const int xa = min(max(x0, 0), qnx - 1), xb = min(max(x0 + 1, 0), qnx - 1);
        const int za = min(max(z0, 0), qnz - 1), zb = min(max(z0 + 1, 0), qnz - 1);
        const long long q_probe = (long long)qnx * qnz;
        const float* up = P.upper + (size_t)bq * (size_t)(4 * P.n_dir) * q_probe * W;
        const int qs[4] = {za * qnx + xa, za * qnx + xb, zb * qnx + xa, zb * qnx + xb};
        const float ws[4] = {(1.0f - fz) * (1.0f - fx), (1.0f - fz) * fx, fz * (1.0f - fx), fz * fx};
#pragma unroll
        for (int w = 0; w < W; ++w) R[w] = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float m[W];
#pragma unroll
            for (int w = 0; w < W; ++w) m[w] = 0.0f;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float* src = up + ((size_t)(4 * k + s) * q_probe + qs[c]) * W;
#pragma unroll
                for (int w = 0; w < W; ++w) m[w] += __ldg(src + w);
            }
#pragma unroll
            for (int w = 0; w < W; ++w) R[w] = fmaf(ws[c] * 0.25f, m[w], R[w]);
        }
    }
    float* dst = P.out + ((size_t)bq * (size_t)P.n_dir * n_probe + (size_t)k * n_probe + p) * W;
#pragma unroll
    for (int w = 0; w < W; ++w) dst[w] = fmaf(T[q * W + w], R[w], I[q * W + w]);
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)nseg);
}

// J at every cell of every non-empty block: the mean of the cascade-0 radiance
// over its n0 directions
template <int W>
__global__ void __launch_bounds__(256) k_rc_mean(const RcParams P, const float* __restrict__ L0, float* __restrict__ J)
{
    const int b = blockIdx.y;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_cells = (long long)P.nx * P.nz;
    if (c >= n_cells) return;
    const int x = (int)(c % P.nx), z = (int)(c / P.nx);
    if (rc_block_state(P.words + (size_t)b * P.n_words, (z >> 4) * P.nbx + (x >> 4)) == 0) return;
    float acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0.0f;
    const float* src = L0 + (size_t)b * (size_t)P.n_dir * n_cells * W;
    for (int k = 0; k < P.n_dir; ++k)
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] += src[((size_t)k * n_cells + c) * W + w];
    const float inv = 1.0f / (float)P.n_dir;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int l = b * W + w;
        if (l < P.n_lambda) J[(size_t)l * n_cells + c] = acc[w] * inv;
    }
}

template <int W, int ST, int NB>
void launch_rc_nb(cudaStream_t s, const RcParams& P, int n_units)
{
    if (n_units == 0) return;
    const long long n = (long long)P.pnx * P.pnz * P.n_dir;
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_units);
    if (P.seg_count) k_rc_cascade<W, true, ST, NB><<<grid, 256, 0, s>>>(P);
    else k_rc_cascade<W, false, ST, NB><<<grid, 256, 0, s>>>(P);
}

template <int W, int ST>
void launch_rc_w(cudaStream_t s, const RcParams& P)
{
    if constexpr (W == 8) {
        if (P.paired) {
            // pairs of batches on one walk each, then the lone batches
            launch_rc_nb<8, ST, 2>(s, P, pair_count(P.n_batch, P.pair_group));
            launch_rc_nb<8, ST, 1>(s, P, pair_lone_count(P.n_batch, P.pair_group));
            return;
        }
    }
    launch_rc_nb<W, ST, 1>(s, P, P.n_batch);
}

}  // namespace

cudaError_t launch_rc_cascade(cudaStream_t s, const RcParams& P)
{
    if (P.n_batch == 0 || P.n_dir == 0) return cudaSuccess;
    switch (P.W * 4 + P.storage) {
        case 1 * 4 + kStoreF32: launch_rc_w<1, kStoreF32>(s, P); break;
        case 2 * 4 + kStoreF32: launch_rc_w<2, kStoreF32>(s, P); break;
        case 4 * 4 + kStoreF32: launch_rc_w<4, kStoreF32>(s, P); break;
        case 8 * 4 + kStoreF32: launch_rc_w<8, kStoreF32>(s, P); break;
        case 8 * 4 + kStoreBF16: launch_rc_w<8, kStoreBF16>(s, P); break;
        case 8 * 4 + kStoreF16: launch_rc_w<8, kStoreF16>(s, P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rc_mean(cudaStream_t s, const RcParams& P, const float* L0, float* J)
{
    if (P.n_batch == 0) return cudaSuccess;
    const long long n_cells = (long long)P.nx * P.nz;
    const dim3 grid((unsigned)((n_cells + 255) / 256), (unsigned)P.n_batch);
    switch (P.W) {
        case 1: k_rc_mean<1><<<grid, 256, 0, s>>>(P, L0, J); break;
        case 2: k_rc_mean<2><<<grid, 256, 0, s>>>(P, L0, J); break;
        case 4: k_rc_mean<4><<<grid, 256, 0, s>>>(P, L0, J); break;
        case 8: k_rc_mean<8><<<grid, 256, 0, s>>>(P, L0, J); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dex
