/*
 * CPU float64 oracle for the plain formal solution on a 3D grid of unit cubic
 * voxels (long characteristics), the three-dimensional form of lc_dense.c.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the product path never
 * does.  It shares no code with the CUDA kernels.
 *
 * What it computes (Section 1, Eq. RteIntegral, piecewise-constant eta and chi
 * per voxel; Section 2.3: the method generalises to 3D with cubic blocks):
 *   the ray p(t) = p_c + t d from a cell centre p_c, t in [0, t_exit], is cut
 *   by every grid plane of the three axes it crosses; each piece lies in one
 *   voxel (found from its midpoint) and is integrated upwind, boundary -> probe:
 *       I <- I exp(-chi l) + (eta / chi) (1 - exp(-chi l))   (I <- I + eta l if chi = 0)
 *   J = sum_k w_k I_k.  Grid layout [nz][ny][nx], x fastest.
 * The pieces come from all plane crossings, sorted (the definition), not from
 * the incremental DDA the GPU uses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double exit3(double o, double d, int n)
{
    if (d > 0.0) return ((double)n - o) / d;
    if (d < 0.0) return (0.0 - o) / d;
    return INFINITY;
}

static int crossings3(double o, double d, int n, double t_exit, double* t, int cap)
{
    int cnt = 0;
    if (d > 0.0) {
        for (long X = (long)floor(o) + 1; X < n; ++X) {
            double tt = ((double)X - o) / d;
            if (tt >= t_exit) break;
            if (tt > 0.0 && cnt < cap) t[cnt++] = tt;
        }
    } else if (d < 0.0) {
        for (long X = (long)ceil(o) - 1; X > 0; --X) {
            double tt = ((double)X - o) / d;
            if (tt >= t_exit) break;
            if (tt > 0.0 && cnt < cap) t[cnt++] = tt;
        }
    }
    return cnt;
}

static long clampl(long v, long n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

/* Pieces of the ray from (ox, oy, oz) along (dx, dy, dz), origin outward:
 * cell[s] = (k * ny + j) * nx + i, len[s] = length.  Zero-length pieces at
 * exact edge/corner crossings are dropped.  Returns the count or -1. */
int oracle3_ray_segments(int nx, int ny, int nz, double ox, double oy, double oz, double dx, double dy, double dz,
                         int cap, int* cell, double* len)
{
    double tex = fmin(fmin(exit3(ox, dx, nx), exit3(oy, dy, ny)), exit3(oz, dz, nz));
    if (!(tex > 0.0) || !isfinite(tex)) return 0;
    int capa = nx + ny + nz + 4;
    double* tx = (double*)malloc(sizeof(double) * (size_t)capa);
    double* ty = (double*)malloc(sizeof(double) * (size_t)capa);
    double* tz = (double*)malloc(sizeof(double) * (size_t)capa);
    int n1 = crossings3(ox, dx, nx, tex, tx, capa);
    int n2 = crossings3(oy, dy, ny, tex, ty, capa);
    int n3 = crossings3(oz, dz, nz, tex, tz, capa);
    double ta = 0.0;
    int a = 0, b = 0, c = 0, ns = 0;
    for (;;) {
        double va = a < n1 ? tx[a] : INFINITY, vb = b < n2 ? ty[b] : INFINITY, vc = c < n3 ? tz[c] : INFINITY;
        double tb;
        if (va <= vb && va <= vc && a < n1) tb = tx[a++];
        else if (vb <= vc && b < n2) tb = ty[b++];
        else if (c < n3) tb = tz[c++];
        else tb = tex;
        if (tb > ta) {
            double mid = 0.5 * (ta + tb);
            long i = clampl((long)floor(ox + mid * dx), nx);
            long j = clampl((long)floor(oy + mid * dy), ny);
            long k = clampl((long)floor(oz + mid * dz), nz);
            if (ns >= cap) { ns = -1; break; }
            cell[ns] = (int)((k * ny + j) * nx + i);
            len[ns] = tb - ta;
            ++ns;
            ta = tb;
        }
        if (tb >= tex) break;
    }
    free(tx);
    free(ty);
    free(tz);
    return ns;
}

static void origin3(int c, int nx, int ny, double* o)
{
    o[0] = (double)(c % nx) + 0.5;
    o[1] = (double)((c / nx) % ny) + 0.5;
    o[2] = (double)(c / (nx * ny)) + 0.5;
}

int64_t oracle3_count_segments(int nx, int ny, int nz, int n_dir, const double* dirs, int n_probe, const int* probes)
{
    int64_t total = 0;
    int cap = 3 * (nx + ny + nz) + 8;
#pragma omp parallel reduction(+ : total)
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int p = 0; p < n_probe; ++p) {
            double o[3];
            origin3(probes[p], nx, ny, o);
            for (int q = 0; q < n_dir; ++q) {
                int ns = oracle3_ray_segments(nx, ny, nz, o[0], o[1], o[2], dirs[3 * q], dirs[3 * q + 1],
                                              dirs[3 * q + 2], cap, cell, len);
                if (ns > 0) total += ns;
            }
        }
        free(cell);
        free(len);
    }
    return total;
}

/* Upwind integration of one wavelength over the pieces, with a per-piece
 * accessor of (eta, chi). */
static double integrate3(int ns, const int* cell, const double* len, const double* el, const double* cl, double i_bc)
{
    double inten = i_bc;
    for (int s = ns - 1; s >= 0; --s) {
        double x = cl[cell[s]], e = el[cell[s]];
        if (x > 0.0) {
            double tau = x * len[s];
            inten = inten * exp(-tau) + (e / x) * (-expm1(-tau));
        } else {
            inten = inten + e * len[s];
        }
    }
    return inten;
}

/*
 * Plain formal solution in 3D.
 *   eta, chi : [n_lambda][nz][ny][nx] float64 per unit length
 *   dirs     : [n_dir][3] unit ray directions, weights [n_dir]
 *   probes   : [n_probe] cell indices (ray origins at their centres)
 *   J        : [n_lambda][n_probe]; I optional [n_lambda][n_dir][n_probe]
 */
int oracle3_formal_solve(int nx, int ny, int nz, int n_lambda, const double* eta, const double* chi, int n_dir,
                         const double* dirs, const double* weights, int n_probe, const int* probes, double i_bc,
                         double* J, double* I)
{
    int cap = 3 * (nx + ny + nz) + 8;
    size_t vol = (size_t)nx * ny * nz;
    int err = 0;
#pragma omp parallel
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < n_probe; ++p) {
            double o[3];
            origin3(probes[p], nx, ny, o);
            for (int l = 0; l < n_lambda; ++l) J[(size_t)l * n_probe + p] = 0.0;
            for (int q = 0; q < n_dir; ++q) {
                int ns = oracle3_ray_segments(nx, ny, nz, o[0], o[1], o[2], dirs[3 * q], dirs[3 * q + 1],
                                              dirs[3 * q + 2], cap, cell, len);
                if (ns < 0) {
#pragma omp atomic write
                    err = 1;
                    ns = 0;
                }
                for (int l = 0; l < n_lambda; ++l) {
                    double inten = integrate3(ns, cell, len, eta + (size_t)l * vol, chi + (size_t)l * vol, i_bc);
                    J[(size_t)l * n_probe + p] += weights[q] * inten;
                    if (I) I[((size_t)l * n_dir + q) * n_probe + p] = inten;
                }
            }
        }
        free(cell);
        free(len);
    }
    return err ? -1 : 0;
}

/*
 * Formal solution over a 3D mipmapped grid with a distance-limited level per
 * block visit (the long-characteristics form of Section 4.1's per-cascade
 * limit): a block first entered at ray parameter t is sampled at level
 * min(L_block, #{band[m-1] <= t}).
 *   lev_eta, lev_chi : the levels 0..n_lev-1 one after the other, level m as
 *                      [n_lambda][nz >> m][ny >> m][nx >> m] (the voxel of level m
 *                      holding cell (i, j, k) is (i >> m, j >> m, k >> m))
 *   block_level      : [n_batch][nbz][nby][nbx] (-1 = empty block)
 */
int oracle3_formal_solve_banded(int nx, int ny, int nz, int n_lambda, int n_lev, const double* lev_eta,
                                const double* lev_chi, const int* block_level, int block, int lambda_batch,
                                int n_band, const double* band, int n_dir, const double* dirs,
                                const double* weights, int n_probe, const int* probes, double i_bc, double* J,
                                double* I)
{
    int cap = 3 * (nx + ny + nz) + 8;
    int nbx = nx / block, nby = ny / block, nbz = nz / block;
    size_t nb = (size_t)nbx * nby * nbz;
    size_t lev_off[8];
    size_t off = 0;
    if (n_lev < 1 || n_lev > 8) return -1;
    for (int m = 0; m < n_lev; ++m) {
        lev_off[m] = off;
        off += (size_t)n_lambda * (size_t)(nz >> m) * (size_t)(ny >> m) * (size_t)(nx >> m);
    }
    int err = 0;
#pragma omp parallel
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
        int* mcap = (int*)malloc(sizeof(int) * (size_t)cap);
        int* blks = (int*)malloc(sizeof(int) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < n_probe; ++p) {
            double o[3];
            origin3(probes[p], nx, ny, o);
            for (int l = 0; l < n_lambda; ++l) J[(size_t)l * n_probe + p] = 0.0;
            for (int q = 0; q < n_dir; ++q) {
                int ns = oracle3_ray_segments(nx, ny, nz, o[0], o[1], o[2], dirs[3 * q], dirs[3 * q + 1],
                                              dirs[3 * q + 2], cap, cell, len);
                if (ns < 0) {
#pragma omp atomic write
                    err = 1;
                    ns = 0;
                }
                double t = 0.0, t_entry = 0.0;
                int prev = -1;
                for (int s = 0; s < ns; ++s) {
                    int c = cell[s];
                    int bi = (c % nx) / block, bj = ((c / nx) % ny) / block, bk = (c / (nx * ny)) / block;
                    int blk = (bk * nby + bj) * nbx + bi;
                    if (blk != prev) { t_entry = t; prev = blk; }
                    int m = 0;
                    while (m < n_band && band[m] <= t_entry) ++m;
                    mcap[s] = m;
                    blks[s] = blk;
                    t += len[s];
                }
                for (int l = 0; l < n_lambda; ++l) {
                    const int* lmap = block_level + (size_t)(l / lambda_batch) * nb;
                    double inten = i_bc;
                    for (int s = ns - 1; s >= 0; --s) {
                        int L = lmap[blks[s]];
                        if (L < 0) continue;
                        int m = L < mcap[s] ? L : mcap[s];
                        if (m >= n_lev) m = n_lev - 1;
                        int c = cell[s];
                        int ci = (c % nx) >> m, cj = ((c / nx) % ny) >> m, ck = (c / (nx * ny)) >> m;
                        size_t idx = lev_off[m] +
                                     (((size_t)l * (nz >> m) + ck) * (size_t)(ny >> m) + cj) * (size_t)(nx >> m) + ci;
                        double x = lev_chi[idx], e = lev_eta[idx];
                        if (x > 0.0) {
                            double tau = x * len[s];
                            inten = inten * exp(-tau) + (e / x) * (-expm1(-tau));
                        } else {
                            inten = inten + e * len[s];
                        }
                    }
                    J[(size_t)l * n_probe + p] += weights[q] * inten;
                    if (I) I[((size_t)l * n_dir + q) * n_probe + p] = inten;
                }
            }
        }
        free(cell);
        free(len);
        free(mcap);
        free(blks);
    }
    return err ? -1 : 0;
}
