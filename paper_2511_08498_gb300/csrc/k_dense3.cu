// Plain full-resolution formal solver on a 3D grid: long characteristics
// (Section 1) from every probe cell centre through the [nz][ny][nx] grid with
// the three-axis Amanatides & Woo DDA, Eq. RteIntegral per voxel segment.
//
// Thread = (probe, wavelength batch), looping over the quadrature so that
// J = sum_k w_k I_k stays in registers; consecutive threads hold consecutive
// probes (neighbouring cells along x for the all-cell solve).  Registers are
// bounded for 3 CTAs per SM: the solve waits on record loads that miss L2 once
// the planes outgrow it, and the extra resident warps hide that latency.  Records are the
// packed (S, chi) wavelength-batch planes of dex_pack_planes.  Plane parameters
// use the two-float hi + lo form of AxisParam on every axis, so path lengths
// are accurate relative to the segment and the exit plane is hit exactly.
#include "dex_internal.h"

namespace dex {

namespace {

template <int W, bool COUNT>
__global__ void __launch_bounds__(256, 3) k_solve_dense3(const Dense3Params P)
{
    const int b = blockIdx.y;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.n_probe) return;
    long long c = p;
    if (P.probes != nullptr) {
        c = P.probes[p];
        if (c < 0 || c >= P.n_cells) {
            raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
            return;
        }
    }
    const long long nxy = (long long)P.nx * P.ny;
    const int i = (int)(c % P.nx), j = (int)((c / P.nx) % P.ny), k = (int)(c / nxy);

    constexpr int REC = 2 * W;
    const float* __restrict__ base = P.planes + (size_t)b * P.n_cells * REC;
    const float* __restrict__ origin_rec = base + (size_t)c * REC;
    const long long row = (long long)P.nx * REC, slab = nxy * REC;
    const int cap = P.nx + P.ny + P.nz + 4;
    float Jw[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Jw[w] = 0.0f;
    unsigned int nseg = 0;
    bool capped = false;

    for (int q = 0; q < P.quad.n_dir; ++q) {
        const float dx = P.quad.dx[q], dy = P.quad.dy[q], dz = P.quad.dz[q];
        // a zero component counts as positive: its planes sit at t = +inf
        const bool negx = dx < 0.0f, negy = dy < 0.0f, negz = dz < 0.0f;
        const int sx = negx ? -1 : 1, sy = negy ? -1 : 1, sz = negz ? -1 : 1;
        const long long stepx = negx ? -REC : REC, stepy = negy ? -row : row, stepz = negz ? -slab : slab;
        const AxisParam ax = axis_param(dx), ay = axis_param(dy), az = axis_param(dz);
        float Px = negx ? -0.5f : 0.5f, Py = negy ? -0.5f : 0.5f, Pz = negz ? -0.5f : 0.5f;
        const float Ex = negx ? (float)(-i) - 0.5f : (float)(P.nx - i) - 0.5f;
        const float Ey = negy ? (float)(-j) - 0.5f : (float)(P.ny - j) - 0.5f;
        const float Ez = negz ? (float)(-k) - 0.5f : (float)(P.nz - k) - 0.5f;
        const float t2 = fminf(fminf(Ex * ax.ih, Ey * ay.ih), Ez * az.ih);

        int ci = i, cj = j, ck = k;
        const float* rp = origin_rec;
        float th_prev = 0.0f, tl_prev = 0.0f;
        float I[W], T[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
        for (int it = 0;; ++it) {
            const float tnx = Px * ax.ih, tny = Py * ay.ih, tnz = Pz * az.ih;
            const int axis = (tnx <= tny && tnx <= tnz) ? 0 : (tny <= tnz ? 1 : 2);
            const float th = axis == 0 ? tnx : (axis == 1 ? tny : tnz);
            const float Pa = axis == 0 ? Px : (axis == 1 ? Py : Pz);
            const AxisParam aa = axis == 0 ? ax : (axis == 1 ? ay : az);
            const float tl = plane_lo(Pa, aa, th);
            // planes sharing a rounded parameter (an edge or a corner) are ordered by
            // their lo parts; the zero-length step between them is clamped at 0
            const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
            if (it >= cap || (unsigned)ci >= (unsigned)P.nx || (unsigned)cj >= (unsigned)P.ny ||
                (unsigned)ck >= (unsigned)P.nz) {
                capped = true;
                break;
            }
            const Record<W> r = RecFmt<W, kStoreF32>::load(rp);
            segments<W>(r.S, r.chi, len * kNegLog2e, I, T);
            if (COUNT) nseg += (th > th_prev);
            if (th >= t2) break;
            // early termination once every transmission is exactly zero (bit-identical);
            // the counting variant walks every cell
            if (!COUNT && (it & 15) == 15 && all_opaque<W>(T)) break;
            th_prev = th;
            tl_prev = tl;
            // the step on the chosen axis as selects (lanes may step on different axes)
            const bool a0 = axis == 0, a1 = axis == 1, a2 = axis == 2;
            Px = a0 ? Px + (float)sx : Px;
            Py = a1 ? Py + (float)sy : Py;
            Pz = a2 ? Pz + (float)sz : Pz;
            ci += a0 ? sx : 0;
            cj += a1 ? sy : 0;
            ck += a2 ? sz : 0;
            rp += a0 ? stepx : (a1 ? stepy : stepz);
        }
        const float wk = P.quad.w[q];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float Iw = fmaf(T[w], P.i_bc, I[w]);
            Jw[w] = fmaf(wk, Iw, Jw[w]);
            const int l = b * W + w;
            if (P.I != nullptr && l < P.n_lambda) P.I[((size_t)l * P.quad.n_dir + q) * P.n_probe + p] = Iw;
        }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int l = b * W + w;
        if (l < P.n_lambda) P.J[(size_t)l * P.n_probe + p] = Jw[w];
    }
    if (capped) raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
    if (COUNT && P.seg_count != nullptr) atomicAdd(P.seg_count, (unsigned long long)nseg);
}

template <int W>
void launch_dense3_w(dim3 grid, cudaStream_t s, const Dense3Params& P)
{
    if (P.seg_count) k_solve_dense3<W, true><<<grid, 256, 0, s>>>(P);
    else k_solve_dense3<W, false><<<grid, 256, 0, s>>>(P);
}

}  // namespace

cudaError_t launch_solve_dense3(cudaStream_t s, const Dense3Params& P)
{
    if (P.n_probe == 0 || P.n_batch == 0) return cudaSuccess;
    const dim3 grid((unsigned)((P.n_probe + 255) / 256), (unsigned)P.n_batch);
    switch (P.W) {
        case 1: launch_dense3_w<1>(grid, s, P); break;
        case 2: launch_dense3_w<2>(grid, s, P); break;
        case 4: launch_dense3_w<4>(grid, s, P); break;
        case 8: launch_dense3_w<8>(grid, s, P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dex
