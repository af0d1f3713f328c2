// Level populations of a multi-level atom: emissivity/opacity from populations,
// radiative-rate reduction and per-cell statistical equilibrium.
//
//  * k_lte_pops      Boltzmann populations (float64), sum = n_H.
//  * k_atom_eta_chi  Section 2, Eqs. Eta/Chi (complete redistribution) plus a
//                    grey background with Planck source function, float32, per
//                    cell (times the cell size).  One thread per cell, all
//                    wavelengths; the Doppler profile of each line is
//                    renormalised to unit quadrature on the line's samples.
//  * k_rates         Jbar_l = sum_k w_k phi_k J_k per line in float64 (the
//                    profile-weighted mean intensity the radiative rates need).
//  * k_se_solve      rate matrix (radiative + collisional, detailed balance)
//                    and the per-cell statistical-equilibrium solve in float64,
//                    ground row replaced by particle conservation; Gaussian
//                    elimination with partial pivoting.  With rho given, the
//                    downward radiative rate is A rho + B_ul Jbar (the MALI
//                    preconditioned rate, rho = 1 - Psibar, Jbar = Jbar_eff).
//  * k_mali_rates    MALI with same-transition preconditioning and the
//                    diagonal operator of the long-characteristics solve
//                    (Section 4.1, after Rybicki & Hummer 1992): per line and
//                    cell, from the previous populations and their J,
//                      rho      = 1 - Psibar
//                               = sum_k w_k phi_k (E*_k chi_line,k + chi_c,k) / chi_k,
//                      Jbar_eff = sum_k w_k phi_k (J_k - (1 - E*_k) eta_line,k / chi_k)
//                               = sum_k w_k phi_k (Jext_k + (1 - E*_k) eta_c,k / chi_k),
//                    E*_k = 1 - Lambda*_k = sum_d w_d e^{-chi_k l_d}, l_d the
//                    path from the cell centre to its boundary along direction d,
//                    Jext the formal solution with the probe's own-cell emission
//                    left out (J = Jext + (1 - E*) (eta_line + eta_c) / chi).
//                    Both forms avoid a cancellation: 1 - Psibar is not 1 minus a
//                    sum near 1 (the profile has unit quadrature), and Jbar_eff is
//                    not J minus the own-cell term, which in a cell thick at every
//                    sampled frequency is J to float32 precision (that difference
//                    stalled the iteration near 1e-2 in float32).
//  * k_max_rel_change  max over non-empty cells and levels of |new - old| / new.
#include "dex_internal.h"

#include <cmath>

namespace dex {

namespace {

constexpr double kH = 6.62607015e-27;
constexpr double kC = 2.99792458e10;
constexpr double kKB = 1.380649e-16;
constexpr double kAMU = 1.66053906660e-24;
constexpr double kColl = 8.629e-6;
constexpr double kSqrtPi = 1.7724538509055160273;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double planck_nu(double nu, double T)
{
    return 2.0 * kH * nu * nu * nu / (kC * kC) / expm1(kH * nu / (kKB * T));
}

// Doppler width (Hz) of line li at temperature T
__device__ __forceinline__ double doppler_width(const AtomParams& P, int li, double T)
{
    return P.nu0[li] / kC * sqrt(2.0 * kKB * T / (P.atom.mass_amu * kAMU));
}

// Renormalisation 1 / sum_k w_k phi_raw(nu_k) of line li (0 if degenerate)
__device__ double profile_norm(const AtomParams& P, int li, double dnu)
{
    double s = 0.0;
    for (int k = 0; k < P.n_lambda; ++k) {
        if (P.tag[k] != li) continue;
        const double u = (P.nu[k] - P.nu0[li]) / dnu;
        s += P.wq[k] * exp(-u * u) / (kSqrtPi * dnu);
    }
    return s > 0.0 ? 1.0 / s : 0.0;
}

__global__ void k_lte_pops(const AtomParams P, long long n_cells, const float* __restrict__ T_,
                           const float* __restrict__ nh_, double* __restrict__ pops)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const double T = T_[c], nh = nh_[c];
        double w[DEX_MAX_LEVELS], s = 0.0;
        for (int i = 0; i < P.atom.n_level; ++i) {
            w[i] = T > 0.0 ? P.atom.g[i] * exp(-P.atom.energy_erg[i] / (kKB * T)) : 0.0;
            s += w[i];
        }
        for (int i = 0; i < P.atom.n_level; ++i) pops[(long long)i * n_cells + c] = s > 0.0 ? w[i] / s * nh : 0.0;
    }
}

__global__ void k_atom_eta_chi(const AtomParams P, long long n_cells, const float* __restrict__ T_,
                               const float* __restrict__ ne_, const double* __restrict__ pops,
                               float* __restrict__ eta, float* __restrict__ chi)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const double T = T_[c], ne = ne_[c];
        if (!(T > 0.0)) {
            for (int k = 0; k < P.n_lambda; ++k) {
                eta[(long long)k * n_cells + c] = 0.0f;
                chi[(long long)k * n_cells + c] = 0.0f;
            }
            continue;
        }
        double dnu[DEX_MAX_LINES], norm[DEX_MAX_LINES], nlo[DEX_MAX_LINES], nup[DEX_MAX_LINES];
        for (int li = 0; li < P.atom.n_line; ++li) {
            dnu[li] = doppler_width(P, li, T);
            norm[li] = profile_norm(P, li, dnu[li]);
            nlo[li] = pops[(long long)P.atom.line_lower[li] * n_cells + c];
            nup[li] = pops[(long long)P.atom.line_upper[li] * n_cells + c];
        }
        const double chi_c = P.atom.background_sigma * ne;
        for (int k = 0; k < P.n_lambda; ++k) {
            const double nu = P.nu[k];
            double e = chi_c * planck_nu(nu, T), x = chi_c;
            const int li = P.tag[k];
            if (li >= 0) {
                const double u = (nu - P.nu0[li]) / dnu[li];
                const double phi = exp(-u * u) / (kSqrtPi * dnu[li]) * norm[li];
                const double f = kH * nu / (4.0 * kPi) * phi;
                e += f * nup[li] * P.atom.line_A[li];
                x += f * (nlo[li] * P.b_lu[li] - nup[li] * P.b_ul[li]);
            }
            eta[(long long)k * n_cells + c] = (float)(e * P.atom.cell_cm);
            chi[(long long)k * n_cells + c] = (float)(x * P.atom.cell_cm);
        }
    }
}

__global__ void k_rates(const AtomParams P, long long n_cells, const float* __restrict__ T_,
                        const float* __restrict__ J, double* __restrict__ jbar)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const double T = T_[c];
        for (int li = 0; li < P.atom.n_line; ++li) {
            double s = 0.0;
            if (T > 0.0) {
                const double dnu = doppler_width(P, li, T);
                const double norm = profile_norm(P, li, dnu);
                for (int k = 0; k < P.n_lambda; ++k) {
                    if (P.tag[k] != li) continue;
                    const double u = (P.nu[k] - P.nu0[li]) / dnu;
                    const double phi = exp(-u * u) / (kSqrtPi * dnu) * norm;
                    s += P.wq[k] * phi * (double)J[(long long)k * n_cells + c];
                }
            }
            jbar[(long long)li * n_cells + c] = s;
        }
    }
}

__global__ void k_mali_rates(const AtomParams P, const OwnCellOperator O, long long n_cells,
                             const float* __restrict__ T_, const float* __restrict__ ne_,
                             const double* __restrict__ pops, const float* __restrict__ Jext,
                             double* __restrict__ rho, double* __restrict__ jeff)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const double T = T_[c], ne = ne_[c];
        const double chi_c = P.atom.background_sigma * ne * P.atom.cell_cm;
        for (int li = 0; li < P.atom.n_line; ++li) {
            double r = 0.0, je = 0.0;
            if (T > 0.0) {
                const double dnu = doppler_width(P, li, T);
                const double norm = profile_norm(P, li, dnu);
                const double nlo = pops[(long long)P.atom.line_lower[li] * n_cells + c];
                const double nup = pops[(long long)P.atom.line_upper[li] * n_cells + c];
                for (int k = 0; k < P.n_lambda; ++k) {
                    if (P.tag[k] != li) continue;
                    const double nu = P.nu[k];
                    const double u = (nu - P.nu0[li]) / dnu;
                    const double phi = exp(-u * u) / (kSqrtPi * dnu) * norm;
                    const double f = kH * nu / (4.0 * kPi) * phi * P.atom.cell_cm;
                    const double chi_l = f * (nlo * P.b_lu[li] - nup * P.b_ul[li]);
                    const double chi = chi_l + chi_c;
                    if (!(chi > 0.0)) continue;
                    // escape from the own cell, summed over the direction groups
                    const float xf = (float)chi;
                    float es = 0.0f;
                    for (int g = 0; g < O.n; ++g) es = fmaf(O.w[g], expf(-xf * O.ell[g]), es);
                    const double e = (double)es;
                    const double wp = P.wq[k] * phi;
                    const double eta_c = chi_c * planck_nu(nu, T);
                    r += wp * (e * chi_l + chi_c) / chi;
                    je += wp * ((double)Jext[(long long)k * n_cells + c] + (1.0 - e) * eta_c / chi);
                }
            }
            rho[(long long)li * n_cells + c] = r;
            jeff[(long long)li * n_cells + c] = je;
        }
    }
}

// |new - old| / new maximised over non-empty cells and levels; positive doubles
// order as their bit patterns, so the maximum is an integer atomicMax
__global__ void k_max_rel_change(int n_level, long long n_cells, const float* __restrict__ T_,
                                 const double* __restrict__ old_p, const double* __restrict__ new_p,
                                 unsigned long long* __restrict__ out)
{
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        if (!(T_[c] > 0.0f)) continue;
        for (int i = 0; i < n_level; ++i) {
            const double a = old_p[(long long)i * n_cells + c], b = new_p[(long long)i * n_cells + c];
            const double d = b > 0.0 ? fabs(b - a) / b : (a == b ? 0.0 : __longlong_as_double(0x7ff0000000000000LL));
            m = d > m || d != d ? d : m;   // a NaN propagates
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_down_sync(0xffffffffu, m, o);
        m = v > m || v != v ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_se_solve(const AtomParams P, long long n_cells, const float* __restrict__ T_,
                           const float* __restrict__ ne_, const float* __restrict__ nh_,
                           const double* __restrict__ jbar, const double* __restrict__ rho,
                           double* __restrict__ pops)
{
    const int nl = P.atom.n_level;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n_cells;
         c += (long long)gridDim.x * blockDim.x) {
        const double T = T_[c], ne = ne_[c], nh = nh_[c];
        if (!(T > 0.0)) {
            for (int i = 0; i < nl; ++i) pops[(long long)i * n_cells + c] = 0.0;
            continue;
        }
        double R[DEX_MAX_LEVELS][DEX_MAX_LEVELS] = {};  // R[i][j]: rate i -> j
        const double sq = sqrt(T);
        for (int i = 0; i < nl; ++i)
            for (int j = i + 1; j < nl; ++j) {
                const double ups = P.atom.upsilon[i][j];
                if (ups <= 0.0) continue;
                const double dE = P.atom.energy_erg[j] - P.atom.energy_erg[i];
                R[i][j] += ne * kColl / (P.atom.g[i] * sq) * ups * exp(-dE / (kKB * T));
                R[j][i] += ne * kColl / (P.atom.g[j] * sq) * ups;
            }
        for (int li = 0; li < P.atom.n_line; ++li) {
            const int lo = P.atom.line_lower[li], up = P.atom.line_upper[li];
            const double jb = jbar[(long long)li * n_cells + c];
            R[lo][up] += P.b_lu[li] * jb;
            R[up][lo] += P.atom.line_A[li] * (rho ? rho[(long long)li * n_cells + c] : 1.0) + P.b_ul[li] * jb;
        }
        // M n = b: row i = inflow - outflow of level i; row 0 = conservation
        double M[DEX_MAX_LEVELS][DEX_MAX_LEVELS + 1];
        for (int i = 0; i < nl; ++i) {
            for (int j = 0; j <= nl; ++j) M[i][j] = 0.0;
            for (int j = 0; j < nl; ++j)
                if (j != i) {
                    M[i][j] += R[j][i];
                    M[i][i] -= R[i][j];
                }
        }
        for (int j = 0; j < nl; ++j) M[0][j] = 1.0;
        M[0][nl] = nh;
        for (int col = 0; col < nl; ++col) {  // elimination with partial pivoting
            int piv = col;
            for (int r = col + 1; r < nl; ++r)
                if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
            if (piv != col)
                for (int j = 0; j <= nl; ++j) {
                    const double t = M[col][j];
                    M[col][j] = M[piv][j];
                    M[piv][j] = t;
                }
            const double inv = 1.0 / M[col][col];
            for (int r = col + 1; r < nl; ++r) {
                const double f = M[r][col] * inv;
                for (int j = col; j <= nl; ++j) M[r][j] -= f * M[col][j];
            }
        }
        double n[DEX_MAX_LEVELS];
        for (int i = nl - 1; i >= 0; --i) {
            double s = M[i][nl];
            for (int j = i + 1; j < nl; ++j) s -= M[i][j] * n[j];
            n[i] = s / M[i][i];
        }
        for (int i = 0; i < nl; ++i) pops[(long long)i * n_cells + c] = n[i];
    }
}

unsigned grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)(b > 152LL * 16 ? 152LL * 16 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t launch_lte_pops(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T,
                            const float* nh, double* pops)
{
    if (n_cells == 0) return cudaSuccess;
    k_lte_pops<<<grid_for(n_cells), 256, 0, s>>>(P, n_cells, T, nh, pops);
    return cudaGetLastError();
}

cudaError_t launch_atom_eta_chi(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T,
                                const float* ne, const double* pops, float* eta, float* chi)
{
    if (n_cells == 0 || P.n_lambda == 0) return cudaSuccess;
    k_atom_eta_chi<<<grid_for(n_cells), 256, 0, s>>>(P, n_cells, T, ne, pops, eta, chi);
    return cudaGetLastError();
}

cudaError_t launch_rates(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T, const float* J,
                         double* jbar)
{
    if (n_cells == 0) return cudaSuccess;
    k_rates<<<grid_for(n_cells), 256, 0, s>>>(P, n_cells, T, J, jbar);
    return cudaGetLastError();
}

cudaError_t launch_se_solve(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T, const float* ne,
                            const float* nh, const double* jbar, const double* rho, double* pops)
{
    if (n_cells == 0) return cudaSuccess;
    k_se_solve<<<grid_for(n_cells), 128, 0, s>>>(P, n_cells, T, ne, nh, jbar, rho, pops);
    return cudaGetLastError();
}

cudaError_t launch_mali_rates(cudaStream_t s, const AtomParams& P, const OwnCellOperator& O, long long n_cells,
                              const float* T, const float* ne, const double* pops, const float* J, double* rho,
                              double* jeff)
{
    if (n_cells == 0 || P.atom.n_line == 0) return cudaSuccess;
    k_mali_rates<<<grid_for(n_cells), 128, 0, s>>>(P, O, n_cells, T, ne, pops, J, rho, jeff);
    return cudaGetLastError();
}

cudaError_t launch_max_rel_change(cudaStream_t s, int n_level, long long n_cells, const float* T, const double* old_p,
                                  const double* new_p, double* out)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess || n_cells == 0) return e;
    k_max_rel_change<<<grid_for(n_cells), 256, 0, s>>>(n_level, n_cells, T, old_p, new_p,
                                                       reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

}  // namespace dex
