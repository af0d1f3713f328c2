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
