// Hierarchical DDA formal solver with one traversal per ray for several
// wavelength batches (Section 2.3, Algorithm 1; Section 4.1's wavelength
// batches, each with its own block levels).
//
// The per-batch solver (k_hdda.cu) traces every ray once per batch of 8
// wavelengths, so the whole traversal -- plane arithmetic, block crossings,
// level look-ups -- is paid once per batch.  Here one thread carries NB batches
// (8 NB wavelengths) of one probe along a single walk:
//
//  * in each block the walk steps through the voxels of the finest level that
//    any batch still being integrated uses there (the "fine" level; a batch
//    whose transmissions have all underflowed to zero is dropped at the next
//    block face, where its own walk would end);
//  * a batch whose own level is coarser keeps the ray parameter at which it
//    entered its current (coarse) voxel and integrates that voxel once, when the
//    walk leaves it -- on a block face, at the exit, or on a fine plane that is
//    also a plane of the batch's level (the fine index on the stepped axis
//    changes its value >> (level - fine level));
//  * the coarse voxel's length is then the difference of the same two plane
//    parameters the batch's own walk would use (coarse planes are fine planes),
//    so each batch is integrated as at its own level (Eq. RteIntegral with the
//    voxel's constant record), and the executed segments are the per-batch ones.
//
// Which batches share a walk: batch b with batch n_batch - 1 - b (a line's
// wavelength batches lie symmetrically about its centre, so their level maps
// tend to agree and the shared walk rarely steps finer than either needs).
// Measured on the 1024^2 static-line workload (32 wavelengths, 64 directions,
// IoD 1e-2): 234 ms against 199 ms for one walk per batch, J bit-identical.
// The two batches' state (I, T, records: 126 registers) halves the resident
// warps, and with them the latency the per-batch walk hides; consecutive
// batches (290 ms) and four batches per walk (299 ms, 242 registers) are
// slower still.  The per-batch walk therefore stays the default.
//
// Each batch's record is loaded at the top of the step after its voxel began
// (kept in registers while the walk crosses the rest of a coarse voxel), so
// the load's latency is hidden by the step's plane and crossing arithmetic.
// J of the group's wavelengths accumulates in shared memory; block look-ups
// read one shared word per block: rank << 12 | the NB 3-bit states.
#include "hdda.cuh"

namespace dex {

namespace {

constexpr int kMbStateBits = 12;       // up to 4 x 3-bit states below the rank
constexpr int kMbMaxBlocks = 24576;    // shared table of 96 KB at most

// Batch carried in slot q of group g (pairs b, n_batch - 1 - b), or -1.
template <int NB>
__host__ __device__ __forceinline__ int group_batch(int g, int q, int n_batch)
{
    const int pairs = (n_batch + 1) / 2;
    const int p = g * (NB / 2) + (q >> 1);   // pair index
    if (p >= pairs) return -1;
    if ((q & 1) == 0) return p;
    const int b = n_batch - 1 - p;
    return b > p ? b : -1;
}

template <int NB>
__host__ __device__ __forceinline__ int group_count(int n_batch)
{
    const int pairs = (n_batch + 1) / 2;
    return (pairs + NB / 2 - 1) / (NB / 2);
}

// One ray from the centre of cell (i, j) of active block a0 = (bx0, bz0) along d:
// accumulates I, T of the group's present batches (slots in `present`).
template <int NB, int ST, bool COUNT>
__device__ __forceinline__ void trace_ray_mb(const Geo& G, const long long* __restrict__ slot_off, unsigned int present,
                                             int i, int j, int bx0, int bz0, int key0, float dx, float dz,
                                             const int* __restrict__ s_info, float* I, float* T, unsigned int& nseg,
                                             bool& capped)
{
    using BF = BrickFmt<8, ST>;
    constexpr int REC = BF::kRec;
    const int cap = 2 * (G.nx + G.nz) + 64;
    const float ox = (float)i + 0.5f, oz = (float)j + 0.5f;
    const bool negx = dx < 0.0f, negz = dz < 0.0f;
    const int sx = negx ? -1 : 1, sz = negz ? -1 : 1;
    const AxisParam ax = axis_param(dx), az = axis_param(dz);
    const float Ex = negx ? (float)(-i) - 0.5f : (float)(G.nx - i) - 0.5f;
    const float Ez = negz ? (float)(-j) - 0.5f : (float)(G.nz - j) - 0.5f;
    const float t2 = fminf(Ex * ax.ih, Ez * az.ih);

    unsigned int live = present;
    int lev[NB];
    int mip = 4;
    {
        const int c0 = distance_cap(G, 0.0f);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            lev[q] = min(((key0 >> (3 * q)) & 7) - 1, c0);
            if ((live >> q) & 1u) mip = min(mip, lev[q]);
        }
    }
    int vox = 1 << mip, side = DEX_BLOCK >> mip;
    float fvox = (float)vox;
    int bxc = bx0, bzc = bz0;
    int lx = (i - bx0 * DEX_BLOCK) >> mip, lz = (j - bz0 * DEX_BLOCK) >> mip;
    float Px = (float)(bx0 * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
    float Pz = (float)(bz0 * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox - j) - 0.5f;
    const float* rp[NB];
    float th0[NB], tl0[NB];
    Record<8> rec[NB];
    {
        const float* blk = G.batch_base + (size_t)(key0 >> kMbStateBits) * G.chain * REC;
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int m = max(lev[q], 0), sh = max(m - mip, 0);
            rp[q] = blk + slot_off[q] + BF::offset(level_offset(m), lz >> sh, lx >> sh, DEX_BLOCK >> m);
            th0[q] = 0.0f;
            tl0[q] = 0.0f;
        }
    }
    unsigned int fresh = live;  // batches whose current voxel's record is still to be loaded

#pragma unroll 1
    for (int it = 0;; ++it) {
        // records of the voxels entered at the last plane, issued before the step's arithmetic
#pragma unroll
        for (int q = 0; q < NB; ++q)
            if ((fresh >> q) & 1u) rec[q] = BF::load(rp[q], BF::chi_off(DEX_BLOCK >> max(lev[q], 0)));
        const float tnx = Px * ax.ih, tnz = Pz * az.ih;
        const bool on_x = tnx <= tnz;
        const float th = on_x ? tnx : tnz;
        const float tl = plane_lo(on_x ? Px : Pz, on_x ? ax : az, th);
        const bool last = th >= t2;
        const int lold = on_x ? lx : lz;
        const int lnew = lold + (on_x ? sx : sz);
        const bool cross = !last && (unsigned)lnew >= (unsigned)side;
        const bool bend = last || cross;
        // batches whose voxel ends on this plane: a block face, the exit, or a fine
        // plane that is also a plane of the batch's level
        unsigned int ends = 0u;
        float nl2[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int sh = lev[q] - mip;
            nl2[q] = fmaxf((th - th0[q]) + (tl - tl0[q]), 0.0f) * kNegLog2e;
            if (mip >= 0 && ((live >> q) & 1u) && (bend || ((lold >> sh) != (lnew >> sh)))) ends |= 1u << q;
        }
        unsigned int pos = 0u;  // ending voxels of positive length (segment count)
        if (COUNT) {
#pragma unroll
            for (int q = 0; q < NB; ++q) pos |= (th > th0[q] ? 1u : 0u) << q;
        }
        // integrate the voxels that ended on this plane (records loaded at the top)
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if ((ends >> q) & 1u) {
                segments<8>(rec[q].S, rec[q].chi, nl2[q], I + 8 * q, T + 8 * q);
                if (COUNT) nseg += (pos >> q) & 1u;
            }
        }
        if (!last) {
            if (it >= cap) { capped = true; break; }
            if (on_x) { lx = lnew; Px += negx ? -fvox : fvox; }
            else { lz = lnew; Pz += negz ? -fvox : fvox; }
            if (!cross) {
                // the ending batches move to the next voxel of their level inside the block
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    if ((ends >> q) & 1u) {
                        const int row = DEX_BLOCK >> lev[q];
                        rp[q] += on_x ? (negx ? -BF::kX : BF::kX) : (negz ? -row * REC : row * REC);
                        th0[q] = th;
                        tl0[q] = tl;
                    }
                }
            }
        }
        unsigned int next_fresh = ends;
        if (cross) {
            // early termination where the ray enters another block, per batch and for
            // the ray: a batch whose every transmission is exactly zero would only add
            // exact zeros (its own walk ends here, after this segment)
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (((live >> q) & 1u) && all_opaque<8>(T + 8 * q)) live &= ~(1u << q);
            if (live == 0u) break;
            const int bxn = bxc + (on_x ? sx : 0), bzn = bzc + (on_x ? 0 : sz);
            if ((unsigned)bxn >= (unsigned)G.nbx || (unsigned)bzn >= (unsigned)G.nbz) {
                capped = true;
                break;
            }
            const int key = s_info[bzn * G.nbx + bxn];
            int mip_new = -1;
            if (key >= 0) {
                const int dc = distance_cap(G, th);
                mip_new = 4;
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    lev[q] = min(((key >> (3 * q)) & 7) - 1, dc);
                    if ((live >> q) & 1u) mip_new = min(mip_new, lev[q]);   // finest level of the live batches
                }
            }
            if (mip_new == mip) {
                if (on_x) lx = negx ? side - 1 : 0;
                else lz = negz ? side - 1 : 0;
            } else {
                // MIP-0 cell entered: exact on the stepped axis, from p(t) on the
                // other one, clamped to the voxel just left
                const int vox_old = vox;
                int m0x, m0z;
                if (on_x) {
                    m0x = bxn * DEX_BLOCK + (negx ? DEX_BLOCK - 1 : 0);
                    const int lo = bzc * DEX_BLOCK + lz * vox_old;
                    m0z = min(max(__float2int_rd(fmaf(th, dz, oz)), lo), lo + vox_old - 1);
                } else {
                    m0z = bzn * DEX_BLOCK + (negz ? DEX_BLOCK - 1 : 0);
                    const int lo = bxc * DEX_BLOCK + lx * vox_old;
                    m0x = min(max(__float2int_rd(fmaf(th, dx, ox)), lo), lo + vox_old - 1);
                }
                mip = mip_new;
                const int shift = mip >= 0 ? mip : 4;
                vox = 1 << shift;
                fvox = (float)vox;
                side = DEX_BLOCK >> shift;
                lx = (m0x - bxn * DEX_BLOCK) >> shift;
                lz = (m0z - bzn * DEX_BLOCK) >> shift;
                Px = (float)(bxn * DEX_BLOCK + (lx + (negx ? 0 : 1)) * vox - i) - 0.5f;
                Pz = (float)(bzn * DEX_BLOCK + (lz + (negz ? 0 : 1)) * vox - j) - 0.5f;
            }
            bxc = bxn;
            bzc = bzn;
            next_fresh = 0u;
            if (mip >= 0) {
                const float* blk = G.batch_base + (size_t)(key >> kMbStateBits) * G.chain * REC;
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const int m = max(lev[q], 0), sh = max(m - mip, 0);
                    rp[q] = blk + slot_off[q] + BF::offset(level_offset(m), lz >> sh, lx >> sh, DEX_BLOCK >> m);
                }
                next_fresh = live;
            }
        }
        if (last) break;
        if (cross) {
#pragma unroll
            for (int q = 0; q < NB; ++q) { th0[q] = th; tl0[q] = tl; }
        }
        fresh = next_fresh;
    }
}

// Grid (capacity, groups); CTA = one active block's 256 probes for the batches of
// group blockIdx.y.  Dynamic shared memory: one int per block.
template <int NB, int ST, bool COUNT>
__global__ void __launch_bounds__(256, 2) k_solve_hdda_mb(const HddaParams P)
{
    extern __shared__ int s_info[];
    __shared__ float s_J[NB * 8][256];
    const int a0 = blockIdx.x;
    if (a0 >= *P.n_active) return;
    const int g = blockIdx.y;
    int bq[NB];
    unsigned int present = 0u;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        bq[q] = group_batch<NB>(g, q, P.n_batch);
        if (bq[q] >= 0) present |= 1u << q;
    }
    const int tid = threadIdx.x;
    const int n_blocks = P.nbx * P.nbz;
    for (int c = tid; c < n_blocks; c += blockDim.x) {
        const int off = P.block_offset[c];
        int key = -1;  // empty: negative
        if (off >= 0) {
            key = off << kMbStateBits;
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (bq[q] >= 0) key |= block_state(P.words + (size_t)bq[q] * P.n_words, c) << (3 * q);
        }
        s_info[c] = key;
    }
#pragma unroll
    for (int w = 0; w < NB * 8; ++w) s_J[w][tid] = 0.0f;
    __syncthreads();

    const int blk0 = P.active[a0];
    const int bx0 = blk0 % P.nbx, bz0 = blk0 / P.nbx;
    const int wrp = tid >> 5;
    const int i = bx0 * DEX_BLOCK + (wrp & 1) * 8 + (tid & 7);
    const int j = bz0 * DEX_BLOCK + (wrp >> 1) * 4 + ((tid & 31) >> 3);
    const int key0 = s_info[blk0];
    bool bad = key0 < 0 || (key0 >> kMbStateBits) != a0;
#pragma unroll
    for (int q = 0; q < NB; ++q) bad = bad || (bq[q] >= 0 && ((key0 >> (3 * q)) & 7) == 0);
    if (bad) {  // the state words do not describe this active block
        raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
        return;
    }
    constexpr int REC = RecFmt<8, ST>::kStride;
    Geo G;
    G.nx = P.nx;
    G.nz = P.nz;
    G.nbx = P.nbx;
    G.nbz = P.nbz;
    G.chain = P.chain;
    G.cap_active = P.cap_active;
    G.batch_base = P.bricks;
    set_box_full(G);
#pragma unroll
    for (int q = 0; q < 4; ++q) G.band[q] = P.band[q];
    long long slot_off[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) slot_off[q] = (long long)max(bq[q], 0) * P.cap_active * P.chain * REC;
    unsigned int nseg = 0;
    bool capped = false;

    for (int k = 0; k < P.quad.n_dir; ++k) {
        const float dx = P.quad.dx[k], dz = P.quad.dz[k];
        float I[NB * 8], T[NB * 8];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                I[8 * q + w] = 0.0f;
                T[8 * q + w] = (present >> q) & 1u ? 1.0f : 0.0f;  // absent slots count as opaque
            }
        }
        trace_ray_mb<NB, ST, COUNT>(G, slot_off, present, i, j, bx0, bz0, key0, dx, dz, s_info, I, T, nseg,
                                    capped);
        const float wk = P.quad.w[k];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const float Iw = fmaf(T[8 * q + w], P.i_bc, I[8 * q + w]);
                s_J[8 * q + w][tid] = fmaf(wk, Iw, s_J[8 * q + w][tid]);
                const int l = bq[q] * 8 + w;
                if (P.I != nullptr && bq[q] >= 0 && l < P.n_lambda)
                    P.I[((size_t)l * P.quad.n_dir + k) * P.n_cells + (size_t)j * P.nx + i] = Iw;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int l = bq[q] * 8 + w;
            if (bq[q] >= 0 && l < P.n_lambda) P.J[(size_t)l * P.n_cells + (size_t)j * P.nx + i] = s_J[8 * q + w][tid];
        }
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)nseg);
}

constexpr int kMbBatches = 2;  // batches per walk

template <int ST>
cudaError_t launch_mb(cudaStream_t s, const HddaParams& P)
{
    const size_t smem = sizeof(int) * (size_t)P.nbx * P.nbz;
    dim3 grid((unsigned)P.cap_active, (unsigned)group_count<kMbBatches>(P.n_batch));
    auto kernel = P.seg_count ? k_solve_hdda_mb<kMbBatches, ST, true> : k_solve_hdda_mb<kMbBatches, ST, false>;
    if (smem > 16 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 256, smem, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

bool solve_hdda_shared_applies(const HddaParams& P)
{
    const long long n_blocks = (long long)P.nbx * P.nbz;
    return P.traversal == DEX_TRAVERSAL_SHARED && !P.exclude_own && P.W == 8 && P.n_batch >= 2 && n_blocks <= kMbMaxBlocks &&
           P.cap_active < (1 << (31 - kMbStateBits));
}

cudaError_t launch_solve_hdda_shared(cudaStream_t s, const HddaParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    switch (P.storage) {
        case kStoreF32: return launch_mb<kStoreF32>(s, P);
        case kStoreBF16: return launch_mb<kStoreBF16>(s, P);
        case kStoreF16: return launch_mb<kStoreF16>(s, P);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dex
