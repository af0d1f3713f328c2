/*
 * CPU float64 oracle for the radiance intervals of one radiance cascade on a 2D
 * grid of unit square voxels.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the product path never
 * does.  It shares no code with the CUDA kernels.
 *
 * What it computes (the radiance-cascade formal solution the paper's code
 * builds around its traversal, Section 4.1 "Model Configuration"): cascade i has
 * probes on a lattice of spacing s = 2^i (probe (px, pz) at (s(px + 1/2),
 * s(pz + 1/2))) and, for each probe and direction d_k, the radiance interval
 * t in [t_s, t_e] of the ray p(t) = p + t d, clipped at the grid boundary.  The
 * ray's voxel pieces come from lc_dense.c (all plane crossings, sorted); the
 * pieces overlapping the interval are integrated upwind from its far end:
 *     I <- I exp(-chi l) + (eta / chi)(1 - exp(-chi l))   (I <- I + eta l if chi = 0)
 *     T <- T exp(-chi l)
 * starting from I = 0, T = 1, so that I is the radiance emitted inside the
 * interval arriving at t_s and T its transmission.  term = 1 when the ray
 * leaves the grid before t_e (the boundary, not the next cascade, lies beyond).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_ray_segments(int nx, int nz, double ox, double oz, double dx, double dz, int cap, int* cell, double* len);

/*
 *   eta, chi : [n_lambda][nz][nx]
 *   dirs     : [n_dir][2] (d_x, d_z)
 *   I, T     : [n_dir][pnz][pnx][n_lambda] outputs, pnx = nx / spacing, pnz = nz / spacing
 *   term     : [n_dir][pnz][pnx] output
 */
int oracle_rc_intervals(int nx, int nz, int n_lambda, const double* eta, const double* chi, int spacing,
                        int n_dir, const double* dirs, double t_s, double t_e, double* I, double* T,
                        unsigned char* term)
{
    const int pnx = nx / spacing, pnz = nz / spacing;
    const long np = (long)pnx * pnz;
    const size_t vol = (size_t)nx * nz;
    const int cap = 2 * (nx + nz) + 8;
    int err = 0;
#pragma omp parallel
    {
        int* cell = (int*)malloc(sizeof(int) * (size_t)cap);
        double* len = (double*)malloc(sizeof(double) * (size_t)cap);
        double* t0 = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < (long)n_dir * np; ++r) {
            const int k = (int)(r / np);
            const long p = r % np;
            const double ox = spacing * ((double)(p % pnx) + 0.5), oz = spacing * ((double)(p / pnx) + 0.5);
            int ns = oracle_ray_segments(nx, nz, ox, oz, dirs[2 * k], dirs[2 * k + 1], cap, cell, len);
            if (ns < 0) {
#pragma omp atomic write
                err = 1;
                ns = 0;
            }
            double t_exit = 0.0;
            for (int s = 0; s < ns; ++s) {
                t0[s] = t_exit;
                t_exit += len[s];
            }
            term[r] = t_exit <= t_e ? 1 : 0;
            for (int l = 0; l < n_lambda; ++l) {
                double inten = 0.0, tr = 1.0;
                for (int s = ns - 1; s >= 0; --s) {
                    const double a = fmax(t0[s], t_s), b = fmin(t0[s] + len[s], t_e);
                    if (!(b > a)) continue;
                    const double ll = b - a;
                    const double x = chi[(size_t)l * vol + (size_t)cell[s]];
                    const double e = eta[(size_t)l * vol + (size_t)cell[s]];
                    if (x > 0.0) {
                        const double tau = x * ll;
                        inten = inten * exp(-tau) + (e / x) * (-expm1(-tau));
                        tr *= exp(-tau);
                    } else {
                        inten += e * ll;
                    }
                }
                I[(size_t)r * n_lambda + l] = inten;
                T[(size_t)r * n_lambda + l] = tr;
            }
        }
        free(cell);
        free(len);
        free(t0);
    }
    return err ? -1 : 0;
}
