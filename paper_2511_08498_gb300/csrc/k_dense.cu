// Plain full-resolution formal solver (long characteristics + Amanatides & Woo DDA)
// and the packing of eta/chi into interleaved wavelength-batch records.
//
// Thread = (probe, wavelength batch).  Each thread walks every quadrature
// direction in turn, so the angular sum J = sum_k w_k I_k stays in registers
// and needs no atomics.  Lanes of a warp hold neighbouring probes and share the
// direction, so their voxels are neighbours in memory and their step counts
// match.  Wavelength batch is the slowest grid dimension so that one batch
// (nx * nz * 8W bytes) is the L2-resident working set at a time.
//
// Plane crossings are evaluated from exact half-integer plane offsets,
//   t_next = offset * fl(1/d)  (+ a low-order part, see AxisParam),
// instead of being accumulated (t += 1/d): every t is within one rounding of
// exact, and the boundary plane's t is bit-identical to the exit parameter, so
// a ray never steps outside the grid.
#include "dex_internal.h"

namespace dex {

namespace {

__global__ void k_pack_planes(long long n_cells, int n_lambda, int W, int n_batch,
                              const float* __restrict__ eta, const float* __restrict__ chi,
                              float* __restrict__ planes, unsigned int* status)
{
    const long long total = n_cells * n_batch;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long c = q % n_cells;
        const int b = (int)(q / n_cells);
        float* rec = planes + q * (2 * W);
        bool bad = false;
        for (int w = 0; w < W; ++w) {
            const int l = b * W + w;
            float S = 0.0f, x = 0.0f;
            if (l < n_lambda) {
                const float e = eta[(long long)l * n_cells + c];
                const float k = chi[(long long)l * n_cells + c];
                if (!(k >= 0.0f) || !(e >= 0.0f) || !isfinite(k) || !isfinite(e) ||
                    (k == 0.0f && e > kEmitterMaxEta)) {
                    bad = true;
                } else {
                    encode_voxel(e, k, S, x);
                }
            }
            rec[w] = S;
            rec[W + w] = x;
        }
        if (bad) raise_status(status, DEX_ERR_NUMERIC);
    }
}

// EXT: the probe's own-cell emission (the first segment of every ray) is left
// out, so I and J hold the radiation arriving from beyond the cell, attenuated
// by it -- the part of J that MALI's effective mean intensity needs without
// subtracting the own-cell term from J (Section 4.1's preconditioning)
template <int W, bool COUNT, bool EXT = false>
__global__ void __launch_bounds__(256, 4) k_solve_dense(const DenseParams P)
{
    const int b = blockIdx.y;
    int i, j, p;
    if (P.probes == nullptr) {  // every cell is a probe
        // 32 x 8 tile of probes per CTA: lanes along x, warps along z
        const int tiles_x = (P.nx + 31) >> 5;
        const int tx = blockIdx.x % tiles_x, tz = blockIdx.x / tiles_x;
        i = tx * 32 + (threadIdx.x & 31);
        j = tz * 8 + (threadIdx.x >> 5);
        if (i >= P.nx || j >= P.nz) return;
        p = j * P.nx + i;
    } else {
        p = blockIdx.x * blockDim.x + threadIdx.x;
        if (p >= P.n_probe) return;
        const int c = P.probes[p];
        if (c < 0 || (long long)c >= P.n_cells) {
            raise_status(P.status, DEX_ERR_TRAVERSAL_CAP);
            return;
        }
        i = c % P.nx;
        j = c / P.nx;
    }

    constexpr int REC = 2 * W;
    const float* __restrict__ base = P.planes + (size_t)b * P.n_cells * REC;
    const float* __restrict__ origin_rec = base + ((size_t)j * P.nx + i) * REC;
    const long long row = (long long)P.nx * REC;
    const int cap = P.nx + P.nz + 4;
    float Jw[W];
#pragma unroll
    for (int w = 0; w < W; ++w) Jw[w] = 0.0f;
    unsigned int nseg = 0;
    bool capped = false;

    for (int k = 0; k < P.quad.n_dir; ++k) {
        const float dx = P.quad.dx[k], dz = P.quad.dz[k];
        // a zero component counts as positive, so its plane offsets are positive
        // and their parameters (offset * inf) are +inf: that axis never steps
        const bool negx = dx < 0.0f, negz = dz < 0.0f;
        const int sx = negx ? -1 : 1, sz = negz ? -1 : 1;
        const float fsx = (float)sx, fsz = (float)sz;
        const long long stepx = negx ? -REC : REC, stepz = negz ? -row : row;
        const AxisParam ax = axis_param(dx), az = axis_param(dz);
        // plane offsets from the origin (half-integers, exact): next plane, exit plane
        float Px = negx ? -0.5f : 0.5f, Pz = negz ? -0.5f : 0.5f;
        const float Ex = negx ? (float)(-i) - 0.5f : (float)(P.nx - i) - 0.5f;
        const float Ez = negz ? (float)(-j) - 0.5f : (float)(P.nz - j) - 0.5f;
        const float t2 = fminf(Ex * ax.ih, Ez * az.ih);

        int ci = i, cj = j;
        const float* rp = origin_rec;
        float th_prev = 0.0f, tl_prev = 0.0f;
        float I[W], T[W];
#pragma unroll
        for (int w = 0; w < W; ++w) { I[w] = 0.0f; T[w] = 1.0f; }
        for (int it = 0;; ++it) {
            if (it >= cap || (unsigned)ci >= (unsigned)P.nx || (unsigned)cj >= (unsigned)P.nz) {
                capped = true;
                break;
            }
            // the record is issued first: the plane arithmetic below hides its latency
            const Record<W> r = RecFmt<W, kStoreF32>::load(rp);
            const float tnx = Px * ax.ih, tnz = Pz * az.ih;
            const bool on_x = tnx <= tnz;
            const float th = on_x ? tnx : tnz;
            const float tl = plane_lo(on_x ? Px : Pz, on_x ? ax : az, th);
            // where an x and a z plane share the rounded parameter (a corner), the lo
            // parts order them and the zero-length step between them can come out a
            // few ulps negative: clamped, or e^{-chi len} overflows in thick cells
            const float len = fmaxf((th - th_prev) + (tl - tl_prev), 0.0f);
            const float nl2 = len * kNegLog2e;
            segments<W>(r.S, r.chi, nl2, I, T);
            if constexpr (EXT) {
                if (it == 0) {
#pragma unroll
                    for (int w = 0; w < W; ++w) I[w] = 0.0f;
                }
            }
            if (COUNT) nseg += (th > th_prev);
            if (th >= t2) break;
            // early termination every 16 cells once every transmission is exactly zero
            // (the rest of the ray would add exact zeros; I and T are unchanged); the
            // counting variant walks every cell: its count is the full-resolution
            // segment count that throughput figures are normalised by
            if (!COUNT && (it & 15) == 15 && all_opaque<W>(T)) break;
            th_prev = th;
            tl_prev = tl;
            if (on_x) { Px += fsx; ci += sx; rp += stepx; }
            else { Pz += fsz; cj += sz; rp += stepz; }
        }
        const float wk = P.quad.w[k];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float Iw = fmaf(T[w], P.i_bc, I[w]);
            Jw[w] = fmaf(wk, Iw, Jw[w]);
            const int l = b * W + w;
            if (P.I != nullptr && l < P.n_lambda)
                P.I[((size_t)l * P.quad.n_dir + k) * P.n_probe + p] = Iw;
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
void launch_dense_w(dim3 grid, cudaStream_t s, const DenseParams& P)
{
    if (P.exclude_own) {
        if (P.seg_count) k_solve_dense<W, true, true><<<grid, 256, 0, s>>>(P);
        else k_solve_dense<W, false, true><<<grid, 256, 0, s>>>(P);
    } else if (P.seg_count) {
        k_solve_dense<W, true><<<grid, 256, 0, s>>>(P);
    } else {
        k_solve_dense<W, false><<<grid, 256, 0, s>>>(P);
    }
}

}  // namespace

cudaError_t launch_pack_planes(cudaStream_t s, long long n_cells, int n_lambda, int W,
                               const float* eta, const float* chi, float* planes, unsigned int* status)
{
    const int n_batch = (n_lambda + W - 1) / W;
    const long long total = n_cells * n_batch;
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    k_pack_planes<<<(unsigned)blocks, 256, 0, s>>>(n_cells, n_lambda, W, n_batch, eta, chi, planes, status);
    return cudaGetLastError();
}

cudaError_t launch_solve_dense(cudaStream_t s, const DenseParams& P)
{
    if (P.n_probe == 0 || P.n_batch == 0) return cudaSuccess;
    dim3 grid;
    if (P.probes == nullptr) {
        const unsigned tiles = (unsigned)(((P.nx + 31) / 32) * ((P.nz + 7) / 8));
        grid = dim3(tiles, (unsigned)P.n_batch);
    } else {
        grid = dim3((unsigned)((P.n_probe + 255) / 256), (unsigned)P.n_batch);
    }
    switch (P.W) {
        case 1: launch_dense_w<1>(grid, s, P); break;
        case 2: launch_dense_w<2>(grid, s, P); break;
        case 4: launch_dense_w<4>(grid, s, P); break;
        case 8: launch_dense_w<8>(grid, s, P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dex
