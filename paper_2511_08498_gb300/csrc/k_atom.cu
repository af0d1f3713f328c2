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
//                    elimination with partial pivoting.
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

__global__ void k_se_solve(const AtomParams P, long long n_cells, const float* __restrict__ T_,
                           const float* __restrict__ ne_, const float* __restrict__ nh_,
                           const double* __restrict__ jbar, double* __restrict__ pops)
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
            R[up][lo] += P.atom.line_A[li] + P.b_ul[li] * jb;
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
                            const float* nh, const double* jbar, double* pops)
{
    if (n_cells == 0) return cudaSuccess;
    k_se_solve<<<grid_for(n_cells), 128, 0, s>>>(P, n_cells, T, ne, nh, jbar, pops);
    return cudaGetLastError();
}

}  // namespace dex
