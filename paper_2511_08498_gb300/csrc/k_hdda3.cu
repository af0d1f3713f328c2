// Hierarchical DDA formal solver over the sparse, mipmapped 3D block grid
// (Section 2.3, Algorithm 1; the paper's adapted grid generalises directly to
// 3D with 8^3 blocks and levels 0..3).
//
// One CTA per (active block, wavelength batch); each thread takes probe cells of
// the 8^3 block in turn, walking every quadrature direction.  The packed 3-bit block
// states of the batch are staged in shared memory when they fit (else read
// through L1 from global memory).
//
// Traversal of one ray p(t) = p_c + t d, as in the 2D solver but on three axes:
//  * within a region of constant voxel size vox = 2^mip (8, the whole block, for
//    an empty block, mip = -1) it is the Amanatides & Woo DDA: the next plane on
//    each axis is the voxel's far face, the nearest one ends the segment;
//  * segments in non-empty blocks are integrated with the voxel's record at
//    level mip; empty blocks are crossed in one step and add nothing;
//  * entering a block at another level re-initialises the tracer: the MIP-0
//    cell entered is exact on the stepped axis and taken from p(t) on the two
//    others, clamped to the voxel just left, then floored to the new voxel size;
//  * a block first entered at ray parameter t uses level
//    min(block level, #{band[m-1] <= t}) (the distance limit).
// Plane parameters are two-float sums (AxisParam), t never decreases and
// lengths are clamped at zero; a ray that would step out of the grid before its
// exit plane sets DEX_ERR_TRAVERSAL_CAP.  (Clipping rays to the box around the
// non-empty blocks, as the 2D solver does, bought nothing on the 256^3 workload
// once the box had to be found in every CTA.)
#include "dex_internal.h"

namespace dex {

namespace {

constexpr int B3 = DEX_BLOCK3;
constexpr int kCells3 = B3 * B3 * B3;
// threads per CTA and the CTAs per SM the register budget targets
constexpr int kThreads3 = 256;
constexpr int kMinBlocks3 = 3;
// state words staged in shared memory up to this many (64 KB); larger grids
// read them from global memory
constexpr int kMaxStagedWords = 8192;

__host__ __device__ constexpr int level_offset3(int m) { return 585 - (585 >> (3 * m)); }

__device__ __forceinline__ int block_state3(const unsigned long long* words, int blk)
{
    const int wi = blk / DEX_STATES_PER_WORD, sh = DEX_STATE_BITS * (blk - wi * DEX_STATES_PER_WORD);
    return (int)((words[wi] >> sh) & 7ull);
}

// A record of zeros (any record format up to 32 floats): integrating it changes
// nothing (tau = 0: 2^x = 1, 1 - e^{-tau} = 0), so rays read it in empty blocks
// instead of branching around the update.
__device__ __align__(32) float g_zero_record3[32] = {0.0f};

// Highest level a block first entered at ray parameter t may use: the number of
// distance thresholds band[m-1] <= t (padded to four by the launcher), and never
// above the chains' top level
__device__ __forceinline__ int distance_cap3(const Hdda3Params& P, float t)
{
    const int m = (P.band[0] <= t) + (P.band[1] <= t) + (P.band[2] <= t) + (P.band[3] <= t);
    return min(m, P.max_mip);
}

// One ray from the centre of cell (i, j, k).  Each step integrates the voxel it
// leaves and steps to the next voxel of the same level; only a step that leaves
// the block (one divergent branch) looks up the next block, after the
// integration.  Block indices change monotonically and a ray takes at most
// 3 * 8 steps in a block, so the grid bounds check also bounds the loop.
//
// NB = 2: the ray carries two wavelength batches whose bricks lie `off` floats
// apart (I, T of 2 W wavelengths, the second batch's from index W); both are
// integrated over every voxel of the walk.
template <int W, bool COUNT, int ST, int NB = 1>
__device__ __forceinline__ void trace_ray3(const Hdda3Params& P, const float* __restrict__ base, long long off,
                                           int i, int j, int k, int bx0, int by0, int bz0, int a0, int mip0, float dx,
                                           float dy, float dz, const unsigned long long* words, float* I, float* T,
                                           unsigned int& nseg, bool& capped)
{
    constexpr int REC = RecFmt<W, ST>::kStride;
    const float ox = (float)i + 0.5f, oy = (float)j + 0.5f, oz = (float)k + 0.5f;
    const bool negx = dx < 0.0f, negy = dy < 0.0f, negz = dz < 0.0f;
    const int sx = negx ? -1 : 1, sy = negy ? -1 : 1, sz = negz ? -1 : 1;
    const AxisParam ax = axis_param(dx), ay = axis_param(dy), az = axis_param(dz);
    const float Ex = negx ? (float)(-i) - 0.5f : (float)(P.nx - i) - 0.5f;
    const float Ey = negy ? (float)(-j) - 0.5f : (float)(P.ny - j) - 0.5f;
    const float Ez = negz ? (float)(-k) - 0.5f : (float)(P.nz - k) - 0.5f;
    const float t2 = fminf(fminf(Ex * ax.ih, Ey * ay.ih), Ez * az.ih);

    // tracer state: level, voxel size, block, block-local voxel, far-face plane offsets
    int mip = mip0, vox = 1 << mip0, side = B3 >> mip0;
    int bxc = bx0, byc = by0, bzc = bz0;
    int lx = (i - bx0 * B3) >> mip, ly = (j - by0 * B3) >> mip, lz = (k - bz0 * B3) >> mip;
    float Px = (float)(bx0 * B3 + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
    float Py = (float)(by0 * B3 + (ly + (negy ? 0 : 1)) * vox - j) - 0.5f;
    float Pz = (float)(bz0 * B3 + (lz + (negz ? 0 : 1)) * vox - k) - 0.5f;
    const float* rp = base + ((size_t)a0 * P.chain + level_offset3(mip) + (lz * side + ly) * side + lx) * REC;
    // the second batch's record (the zero record in empty blocks)
    const float* rp2 = NB == 2 ? rp + off : nullptr;
    float th_prev = 0.0f, tl_prev = 0.0f;

    Record<W> r, r2;
    for (int it = 0;; ++it) {
        // float32 records: issued at the top of the step (256-bit loads), so that the
        // stepping and crossing bookkeeping hides their latency
        if constexpr (ST == kStoreF32) {
            r = RecFmt<W, ST>::load(rp);
            if constexpr (NB == 2) r2 = RecFmt<W, ST>::load(rp2);
        }
        const float tnx = Px * ax.ih, tny = Py * ay.ih, tnz = Pz * az.ih;
        const int axis = (tnx <= tny && tnx <= tnz) ? 0 : (tny <= tnz ? 1 : 2);
        const float th = axis == 0 ? tnx : (axis == 1 ? tny : tnz);
        const float tl = plane_lo(axis == 0 ? Px : (axis == 1 ? Py : Pz), axis == 0 ? ax : (axis == 1 ? ay : az), th);
        const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
        const bool last = th >= t2;
        const int cur_mip = mip;
        const float* cur_rp = rp;
        const float* cur_rp2 = rp2;
        // the step on the chosen axis, written as selects (no divergent branch
        // when the lanes of a warp step on different axes); not used once last
        const float fv = (float)vox;
        const bool a0x = axis == 0, a1 = axis == 1;
        lx += a0x ? sx : 0;
        ly += a1 ? sy : 0;
        lz += (!a0x && !a1) ? sz : 0;
        Px = a0x ? (negx ? Px - fv : Px + fv) : Px;
        Py = a1 ? (negy ? Py - fv : Py + fv) : Py;
        Pz = (!a0x && !a1) ? (negz ? Pz - fv : Pz + fv) : Pz;
        const int st_ax = a0x ? 1 : (a1 ? side : side * side);
        const bool ng = a0x ? negx : (a1 ? negy : negz);
        rp += (ng ? -st_ax : st_ax) * REC;
        if constexpr (NB == 2) rp2 += (ng ? -st_ax : st_ax) * REC;
        const int la = a0x ? lx : (a1 ? ly : lz);
        const bool cross = (unsigned)la >= (unsigned)side;
        // integrate the voxel left (the zero record in empty blocks)
        const float nl2 = len * kNegLog2e;
        if constexpr (ST != kStoreF32) r = RecFmt<W, ST>::template load<false>(cur_rp);
        segments<W>(r.S, r.chi, nl2, I, T);
        if constexpr (NB == 2) {
            if constexpr (ST != kStoreF32) r2 = RecFmt<W, ST>::template load<false>(cur_rp2);
            segments<W>(r2.S, r2.chi, nl2, I + W, T + W);
        }
        if (COUNT) nseg += (cur_mip >= 0) & (th > th_prev);
        if (last) break;
        th_prev = th;
        tl_prev = tl;
        if (cross) {  // entered another block
            // early termination: once every transmission is exactly zero the rest of
            // the ray adds exact zeros (bit-identical)
            if (all_opaque<NB * W>(T)) break;
            const int bxn = bxc + (axis == 0 ? sx : 0), byn = byc + (axis == 1 ? sy : 0),
                      bzn = bzc + (axis == 2 ? sz : 0);
            if ((unsigned)bxn >= (unsigned)P.nbx || (unsigned)byn >= (unsigned)P.nby ||
                (unsigned)bzn >= (unsigned)P.nbz) {
                capped = true;
                break;
            }
            const int blk = (bzn * P.nby + byn) * P.nbx + bxn;
            const int st = block_state3(words, blk) - 1;
            const int mip_new = st < 0 ? -1 : min(st, distance_cap3(P, th));
            if (mip_new == mip) {
                if (axis == 0) lx = negx ? side - 1 : 0;
                else if (axis == 1) ly = negy ? side - 1 : 0;
                else lz = negz ? side - 1 : 0;
            } else {
                // MIP-0 cell entered: exact on the stepped axis, from p(t) on the two
                // others, clamped to the voxel just left
                const int vo = vox;
                const int lox = bxc * B3 + lx * vo, loy = byc * B3 + ly * vo, loz = bzc * B3 + lz * vo;
                const int m0x = axis == 0 ? bxn * B3 + (negx ? B3 - 1 : 0)
                                          : min(max(__float2int_rd(fmaf(th, dx, ox)), lox), lox + vo - 1);
                const int m0y = axis == 1 ? byn * B3 + (negy ? B3 - 1 : 0)
                                          : min(max(__float2int_rd(fmaf(th, dy, oy)), loy), loy + vo - 1);
                const int m0z = axis == 2 ? bzn * B3 + (negz ? B3 - 1 : 0)
                                          : min(max(__float2int_rd(fmaf(th, dz, oz)), loz), loz + vo - 1);
                mip = mip_new;
                const int shift = mip >= 0 ? mip : 3;
                vox = 1 << shift;
                side = B3 >> shift;
                lx = (m0x - bxn * B3) >> shift;
                ly = (m0y - byn * B3) >> shift;
                lz = (m0z - bzn * B3) >> shift;
                Px = (float)(bxn * B3 + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
                Py = (float)(byn * B3 + (ly + (negy ? 0 : 1)) * vox - j) - 0.5f;
                Pz = (float)(bzn * B3 + (lz + (negz ? 0 : 1)) * vox - k) - 0.5f;
            }
            bxc = bxn;
            byc = byn;
            bzc = bzn;
            rp = mip >= 0 ? base + ((size_t)P.block_offset[blk] * P.chain + level_offset3(mip) +
                                    (lz * side + ly) * side + lx) * REC
                          : g_zero_record3;
            if constexpr (NB == 2) rp2 = mip >= 0 ? rp + off : g_zero_record3;
        }
    }
}

// Packed 3-bit states of two batches, state by state the smaller (0 = empty
// wins): the level map of a walk shared by the two.
__device__ __forceinline__ unsigned long long min_states(unsigned long long a, unsigned long long b)
{
    unsigned long long m = 0ull;
#pragma unroll
    for (int q = 0; q < DEX_STATES_PER_WORD; ++q) {
        const int sh = DEX_STATE_BITS * q;
        const unsigned long long sa = (a >> sh) & 7ull, sb = (b >> sh) & 7ull;
        m |= (sa < sb ? sa : sb) << sh;
    }
    return m;
}

// NB = 1: one CTA per (active block, wavelength batch).  NB = 2: one CTA per
// (active block, pair of batches, pair_batches), walking once for both on the
// smaller of their levels (the state words must fit in shared memory).
template <int W, bool COUNT, int ST, int NB>
__global__ void __launch_bounds__(kThreads3, NB == 1 ? kMinBlocks3 : 2) k_solve_hdda3(const Hdda3Params P)
{
    extern __shared__ unsigned long long s_words[];
    __shared__ float s_J3[NB == 2 ? 2 * W : 1][kThreads3];
    const int a0 = blockIdx.x;
    if (a0 >= *P.n_active) return;
    int b = blockIdx.y, b2 = b;
    if constexpr (NB == 2) pair_batches(blockIdx.y, P.n_batch, P.pair_group, b, b2);
    const int tid = threadIdx.x;
    const unsigned long long* gw = P.words + (size_t)b * P.n_words;
    const bool staged = NB == 2 || P.n_words <= kMaxStagedWords;
    if (staged) {
        if constexpr (NB == 2) {
            const unsigned long long* gw2 = P.words + (size_t)b2 * P.n_words;
            for (int q = tid; q < P.n_words; q += kThreads3) s_words[q] = min_states(gw[q], gw2[q]);
        } else {
            for (int q = tid; q < P.n_words; q += kThreads3) s_words[q] = gw[q];
        }
        __syncthreads();
    }
    const unsigned long long* words = staged ? s_words : gw;
    const int blk0 = P.active[a0];
    const int bx0 = blk0 % P.nbx, by0 = (blk0 / P.nbx) % P.nby, bz0 = blk0 / (P.nbx * P.nby);
    const int state0 = block_state3(words, blk0) - 1;
    if (state0 < 0) {  // state words do not describe this active block
        raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
        return;
    }
    constexpr int REC = RecFmt<W, ST>::kStride;
    const size_t batch_floats = (size_t)P.cap_active * P.chain * REC;
    const float* base = P.bricks + (size_t)b * batch_floats;
    const long long off = (long long)(b2 - b) * (long long)batch_floats;
    const int mip0 = min(state0, distance_cap3(P, 0.0f));
    unsigned int nseg = 0;
    bool capped = false;

    // each thread takes kCells3 / kThreads3 probes of the block, one after the other
    for (int pc = tid; pc < kCells3; pc += kThreads3) {
        const int i = bx0 * B3 + (pc & 7), j = by0 * B3 + ((pc >> 3) & 7), k = bz0 * B3 + (pc >> 6);
        const size_t cell = ((size_t)k * P.ny + j) * P.nx + i;
        // J of the probe: registers for one batch, shared memory for a pair (whose
        // I and T take the registers)
        float Jr[NB == 1 ? W : 1];
        auto Jw = [&](int w) -> float& { return NB == 1 ? Jr[NB == 1 ? w : 0] : s_J3[w][tid]; };
#pragma unroll
        for (int w = 0; w < NB * W; ++w) Jw(w) = 0.0f;
        for (int q = 0; q < P.quad.n_dir; ++q) {
            float I[NB * W], T[NB * W];
#pragma unroll
            for (int w = 0; w < NB * W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
            trace_ray3<W, COUNT, ST, NB>(P, base, off, i, j, k, bx0, by0, bz0, a0, mip0, P.quad.dx[q], P.quad.dy[q],
                                         P.quad.dz[q], words, I, T, nseg, capped);
            const float wk = P.quad.w[q];
#pragma unroll
            for (int w = 0; w < NB * W; ++w) {
                const float Iw = fmaf(T[w], P.i_bc, I[w]);
                Jw(w) = fmaf(wk, Iw, Jw(w));
                const int l = w < W ? b * W + w : b2 * W + (w - W);
                if (P.I != nullptr && l < P.n_lambda) P.I[((size_t)l * P.quad.n_dir + q) * P.n_cells + cell] = Iw;
            }
        }
#pragma unroll
        for (int w = 0; w < NB * W; ++w) {
            const int l = w < W ? b * W + w : b2 * W + (w - W);
            if (l < P.n_lambda) P.J[(size_t)l * P.n_cells + cell] = Jw(w);
        }
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    // the walk's segments, once per batch it carries
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)NB * nseg);
}

template <typename K>
cudaError_t launch3(K kernel, dim3 grid, size_t smem, cudaStream_t s, const Hdda3Params& P)
{
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, kThreads3, smem, s>>>(P);
    return cudaSuccess;
}

}  // namespace

bool solve_hdda3_paired_applies(const Hdda3Params& P)
{
    return P.W == 8 && P.n_words <= kMaxStagedWords;
}

cudaError_t launch_solve_hdda3(cudaStream_t s, const Hdda3Params& P0)
{
    // distance thresholds padded to four: +inf beyond n_band, 0 for no limit
    Hdda3Params P = P0;
    for (int q = 0; q < 4; ++q)
        P.band[q] = P0.n_band < 0 ? 0.0f : (q < P0.n_band ? P0.band[q] : __builtin_huge_valf());
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    const size_t smem = P.n_words <= kMaxStagedWords ? sizeof(unsigned long long) * (size_t)P.n_words : 0;
    cudaError_t e = cudaSuccess;
    if (P.traversal == DEX_TRAVERSAL_PAIRED) {
        if (!solve_hdda3_paired_applies(P)) return cudaErrorNotSupported;
        const int n_pairs = pair_count(P.n_batch, P.pair_group);
        if (n_pairs > 0) {
            const dim3 grid2((unsigned)P.cap_active, (unsigned)n_pairs);
            switch (P.storage) {
#define DEX_LAUNCH3P(ST)                                                                     \
    case ST:                                                                                 \
        e = P.seg_count ? launch3(k_solve_hdda3<8, true, ST, 2>, grid2, smem, s, P)          \
                        : launch3(k_solve_hdda3<8, false, ST, 2>, grid2, smem, s, P);        \
        break;
                DEX_LAUNCH3P(kStoreF32)
                DEX_LAUNCH3P(kStoreBF16)
                DEX_LAUNCH3P(kStoreF16)
#undef DEX_LAUNCH3P
                default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // the middle batch of every group of odd size alone, by the per-batch walk
        // on a view of that batch
        for (int q = 0; q < pair_lone_count(P.n_batch, P.pair_group); ++q) {
            const int m = pair_lone_batch(q, P.n_batch, P.pair_group);
            Hdda3Params Q = P0;
            Q.traversal = DEX_TRAVERSAL_PER_BATCH;
            Q.n_batch = 1;
            Q.n_lambda = min(8, P.n_lambda - m * 8);
            Q.bricks = P.bricks + (size_t)m * P.cap_active * P.chain * record_floats(8, P.storage);
            Q.words = P.words + (size_t)m * P.n_words;
            Q.J = P.J + (size_t)m * 8 * P.n_cells;
            Q.I = P.I ? P.I + (size_t)m * 8 * P.quad.n_dir * P.n_cells : nullptr;
            if ((e = launch_solve_hdda3(s, Q)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    switch (P.W * 4 + P.storage) {
#define DEX_LAUNCH3(WW, ST)                                                                 \
    case WW * 4 + ST:                                                                       \
        e = P.seg_count ? launch3(k_solve_hdda3<WW, true, ST, 1>, grid, smem, s, P)         \
                        : launch3(k_solve_hdda3<WW, false, ST, 1>, grid, smem, s, P);       \
        break;
        DEX_LAUNCH3(1, kStoreF32)
        DEX_LAUNCH3(2, kStoreF32)
        DEX_LAUNCH3(4, kStoreF32)
        DEX_LAUNCH3(8, kStoreF32)
        DEX_LAUNCH3(4, kStoreBF16)
        DEX_LAUNCH3(8, kStoreBF16)
        DEX_LAUNCH3(4, kStoreF16)
        DEX_LAUNCH3(8, kStoreF16)
#undef DEX_LAUNCH3
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dex
