/*
 * CPU float64 oracle for the plain formal solution of the radiative transfer
 * equation on a 2D grid of unit square voxels (long characteristics).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the product path never
 * does.  It shares no code with the CUDA kernels.
 *
 * What it computes (Section 1, Eq. RteIntegral, with eta and chi constant in
 * each voxel as in Section 4.1 "Model Configuration"):
 *   For a probe at cell centre p_c and a quadrature direction d, the ray
 *   p(t) = p_c + t d, t in [0, t_exit], is cut by every grid plane it crosses.
 *   Each piece [t_a, t_b] lies inside one voxel i (found from the midpoint),
 *   with path length l_i = t_b - t_a.  The intensity arriving at p_c from the
 *   boundary along this ray is integrated upwind, boundary -> probe:
 *       I <- I exp(-chi_i l_i) + (eta_i / chi_i) (1 - exp(-chi_i l_i))
 *   (I <- I + eta_i l_i when chi_i = 0), starting from I = I_bc.
 *   The mean intensity is J = sum_k w_k I_k (Section 1, angular quadrature).
 *
 * The piece enumeration is the definition written out (all plane crossings,
 * sorted), not the incremental DDA of Amanatides & Woo used on the GPU.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double exit_param(double o, double d, int n)
{
    if (d > 0.0) return ((double)n - o) / d;
    if (d < 0.0) return (0.0 - o) / d;
    return INFINITY;
}

/* Fill t[] with the parameters of the interior planes of one axis crossed for
 * 0 < t < t_exit, in increasing order.  Returns the count. */
static int axis_crossings(double o, double d, int n, double t_exit, double* t, int cap)
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

/*
 * Pieces of the ray p(t) = (ox, oz) + t (dx, dz) inside the nx x nz grid, from
 * the origin outward.  cell[s] = j * nx + i, len[s] = piece length.  Returns
 * the number of pieces (pieces of zero length at exact corner crossings are
 * dropped), or -1 if cap is too small.
 */
int oracle_ray_segments(int nx, int nz, double ox, double oz, double dx, double dz,
                        int cap, int* cell, double* len)
{
    double tex = fmin(exit_param(ox, dx, nx), exit_param(oz, dz, nz));
    if (!(tex > 0.0) || !isfinite(tex)) return 0;
    int cap_axis = nx + nz + 4;
    double* tx = (double*)malloc(sizeof(double) * (size_t)cap_axis);
    double* tz = (double*)malloc(sizeof(double) * (size_t)cap_axis);
    int nxc = axis_crossings(ox, dx, nx, tex, tx, cap_axis);
    int nzc = axis_crossings(oz, dz, nz, tex, tz, cap_axis);
    /* merge the two increasing lists, bracketed by 0 and t_exit */
    double ta = 0.0;
    int a = 0, b = 0, ns = 0;
    for (;;) {
        double tb;
        if (a < nxc && (b >= nzc || tx[a] <= tz[b])) tb = tx[a++];
        else if (b < nzc) tb = tz[b++];
        else tb = tex;
        if (tb > ta) {
            double mid = 0.5 * (ta + tb);
            long i = (long)floor(ox + mid * dx);
            long j = (long)floor(oz + mid * dz);
            if (i < 0) i = 0;
            if (i >= nx) i = nx - 1;
            if (j < 0) j = 0;
            if (j >= nz) j = nz - 1;
            if (ns >= cap) { ns = -1; break; }
            cell[ns] = (int)(j * nx + i);
            len[ns] = tb - ta;
            ++ns;
            ta = tb;
        }
        if (tb >= tex) break;
    }
    free(tx);
    free(tz);
    return ns;
}

/* Number of pieces of every (probe, direction) ray: the dense voxel-segment count. */
int64_t oracle_count_segments(int nx, int nz, int n_dir, const double* dirs,
                              int n_probe, const int* probes)
{
    int64_t total = 0;
    int cap = 2 * (nx + nz) + 8;
#pragma omp parallel reduction(+ : total)
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int p = 0; p < n_probe; ++p) {
            int c = probes[p];
            double ox = (double)(c % nx) + 0.5, oz = (double)(c / nx) + 0.5;
            for (int k = 0; k < n_dir; ++k) {
                int ns = oracle_ray_segments(nx, nz, ox, oz, dirs[2 * k], dirs[2 * k + 1], cap, cell, len);
                if (ns > 0) total += ns;
            }
        }
        free(cell);
        free(len);
    }
    return total;
}

/*
 * Plain formal solution.
 *   eta, chi : [n_lambda][nz][nx] float64, per unit length (cell side = 1)
 *   dirs     : [n_dir][2] (x, z) ray directions, weights: [n_dir]
 *   probes   : [n_probe] cell indices j * nx + i (ray origins at their centres)
 *   J        : [n_lambda][n_probe] output, mean intensity
 *   I        : optional [n_lambda][n_dir][n_probe] output (NULL to skip); I[.][k][.]
 *              is the intensity reaching the probe along the ray traced toward +d_k
 * Returns 0, or -1 on a capacity error.
 */
int oracle_formal_solve(int nx, int nz, int n_lambda, const double* eta, const double* chi,
                        int n_dir, const double* dirs, const double* weights,
                        int n_probe, const int* probes, double i_bc, double* J, double* I)
{
    int cap = 2 * (nx + nz) + 8;
    size_t plane = (size_t)nx * (size_t)nz;
    int err = 0;
#pragma omp parallel
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < n_probe; ++p) {
            int c = probes[p];
            double ox = (double)(c % nx) + 0.5, oz = (double)(c / nx) + 0.5;
            for (int l = 0; l < n_lambda; ++l) J[(size_t)l * n_probe + p] = 0.0;
            for (int k = 0; k < n_dir; ++k) {
                int ns = oracle_ray_segments(nx, nz, ox, oz, dirs[2 * k], dirs[2 * k + 1], cap, cell, len);
                if (ns < 0) {
#pragma omp atomic write
                    err = 1;
                    ns = 0;
                }
                for (int l = 0; l < n_lambda; ++l) {
                    const double* el = eta + (size_t)l * plane;
                    const double* cl = chi + (size_t)l * plane;
                    double inten = i_bc;
                    for (int s = ns - 1; s >= 0; --s) { /* upwind: boundary -> probe */
                        double x = cl[cell[s]], e = el[cell[s]];
                        if (x > 0.0) {
                            double tau = x * len[s];
                            inten = inten * exp(-tau) + (e / x) * (-expm1(-tau));
                        } else {
                            inten = inten + e * len[s];
                        }
                    }
                    J[(size_t)l * n_probe + p] += weights[k] * inten;
                    if (I) I[((size_t)l * n_dir + k) * n_probe + p] = inten;
                }
            }
        }
        free(cell);
        free(len);
    }
    return err ? -1 : 0;
}

/* Threads the OpenMP runtime will use (reported with oracle timings). */
int oracle_num_threads(void)
{
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}

/*
 * Formal solution over a mipmapped grid with a distance-limited level per
 * block visit (Section 4.1: each radiance-cascade interval samples at most a
 * given MIP level, full resolution near the probe and coarser far away; here
 * the long-characteristics form: a block first entered at ray parameter t is
 * sampled at level min(L_block, m_max(t)), m_max(t) = number of thresholds
 * band[m-1] <= t for m = 1..n_band).
 *   lev_eta, lev_chi : [n_lev][n_lambda][nz][nx]; entry [m][l][c] is the value of
 *                      the level-m voxel containing cell c (level 0 = the cell)
 *   block_level      : [n_batch][nbz][nbx] selected level (-1 = empty block)
 *   block, lambda_batch : block side and wavelengths per level map
 * Other arguments as oracle_formal_solve.  Returns 0 or -1.
 */
int oracle_formal_solve_banded(int nx, int nz, int n_lambda, int n_lev, const double* lev_eta,
                               const double* lev_chi, const int* block_level, int block, int lambda_batch,
                               int n_band, const double* band, int n_dir, const double* dirs,
                               const double* weights, int n_probe, const int* probes, double i_bc,
                               double* J, double* I)
{
    int cap = 2 * (nx + nz) + 8;
    size_t plane = (size_t)nx * (size_t)nz;
    int nbx = nx / block, nbz = nz / block;
    int err = 0;
#pragma omp parallel
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
        int* mcap = (int*)malloc(sizeof(int) * (size_t)cap);
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < n_probe; ++p) {
            int c = probes[p];
            double ox = (double)(c % nx) + 0.5, oz = (double)(c / nx) + 0.5;
            for (int l = 0; l < n_lambda; ++l) J[(size_t)l * n_probe + p] = 0.0;
            for (int k = 0; k < n_dir; ++k) {
                int ns = oracle_ray_segments(nx, nz, ox, oz, dirs[2 * k], dirs[2 * k + 1], cap, cell, len);
                if (ns < 0) {
#pragma omp atomic write
                    err = 1;
                    ns = 0;
                }
                /* distance cap of each piece: from the parameter at which its block was entered */
                double t = 0.0, t_entry = 0.0;
                int prev_blk = -1;
                for (int s = 0; s < ns; ++s) {
                    int bi = (cell[s] % nx) / block, bj = (cell[s] / nx) / block;
                    int blk = bj * nbx + bi;
                    if (blk != prev_blk) { t_entry = t; prev_blk = blk; }
                    int m = 0;
                    while (m < n_band && band[m] <= t_entry) ++m;
                    mcap[s] = m;
                    t += len[s];
                }
                for (int l = 0; l < n_lambda; ++l) {
                    const int* lmap = block_level + (size_t)(l / lambda_batch) * nbx * nbz;
                    double inten = i_bc;
                    for (int s = ns - 1; s >= 0; --s) {
                        int bi = (cell[s] % nx) / block, bj = (cell[s] / nx) / block;
                        int L = lmap[bj * nbx + bi];
                        if (L < 0) continue; /* empty block: eta = chi = 0 */
                        int m = L < mcap[s] ? L : mcap[s];
                        if (m >= n_lev) m = n_lev - 1;
                        size_t off = ((size_t)m * n_lambda + l) * plane + (size_t)cell[s];
                        double x = lev_chi[off], e = lev_eta[off];
                        if (x > 0.0) {
                            double tau = x * len[s];
                            inten = inten * exp(-tau) + (e / x) * (-expm1(-tau));
                        } else {
                            inten = inten + e * len[s];
                        }
                    }
                    J[(size_t)l * n_probe + p] += weights[k] * inten;
                    if (I) I[((size_t)l * n_dir + k) * n_probe + p] = inten;
                }
            }
        }
        free(cell);
        free(len);
        free(mcap);
    }
    (void)nbz;
    return err ? -1 : 0;
}
