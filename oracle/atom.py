"""Float64 oracle for the statistical-equilibrium (level population) workload.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

What it computes, in cgs units, cell by cell:

* Section 2, Eqs. Eta and Chi (complete redistribution):
      eta_l = (h nu / 4 pi) n_j A_ji phi(nu),
      chi_l = (h nu / 4 pi) (n_i B_ij - n_j B_ji) phi(nu),
  with B_ji = A_ji c^2 / (2 h nu0^3), B_ij = (g_j / g_i) B_ji; phi a Doppler
  (Gaussian) profile in frequency, Doppler width nu0 / c sqrt(2 k T / m),
  renormalised so that its quadrature over the line's sample points is 1; plus
  a grey background chi_c = sigma n_e with source function B_nu(T) (Planck).
  Opacities and emissivities are per cell (times the cell size).
* Radiative rates from the mean intensity: Jbar = sum_k w_k phi_k J_k over the
  line's frequency points (trapezoid weights in frequency), R_ij = B_ij Jbar,
  R_ji = A_ji + B_ji Jbar.
* Collisional rates: C_ij = n_e 8.629e-6 / (g_i sqrt(T)) Upsilon_ij e^{-dE/kT}
  (i < j) and detailed balance C_ji = C_ij (g_i / g_j) e^{dE/kT}.
* Statistical equilibrium: sum_{j != i} n_j P_ji - n_i sum_{j != i} P_ij = 0
  with P = R + C, the ground-level row replaced by sum_i n_i = n_H; solved
  per cell with numpy.linalg.solve in float64.
* Lambda iteration: LTE (Boltzmann) start, then [eta, chi -> formal solution
  -> J -> rates -> statistical equilibrium] repeated a fixed number of times.
  The paper iterates with MALI (Section 4.1); a plain Lambda iteration of fixed
  length is the workload here.
"""

from __future__ import annotations

import numpy as np

H = 6.62607015e-27
C = 2.99792458e10
K_B = 1.380649e-16
AMU = 1.66053906660e-24
EV = 1.602176634e-12
SIGMA_C = 6.652e-25     # grey background cross-section per electron (cm^2)
COLL = 8.629e-6         # collision-rate constant (cgs)


def planck_nu(nu, T):
    """B_nu(T) (erg s^-1 cm^-2 Hz^-1 sr^-1); 0 where T <= 0."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        x = H * nu / (K_B * T)
        out = 2.0 * H * nu ** 3 / C ** 2 / np.expm1(x)
    return np.where(T > 0, out, 0.0)


def einstein_b(atom):
    """(B_ul, B_lu) per line, frequency units."""
    out = []
    for (lo, up, A, lam0) in atom["lines"]:
        nu0 = C / (lam0 * 1e-7)
        b_ul = A * C ** 2 / (2.0 * H * nu0 ** 3)
        out.append((b_ul, atom["g"][up] / atom["g"][lo] * b_ul))
    return out


def frequency_weights(lam_nm, tag, line):
    """Trapezoid weights in frequency of the sample points of one line (others 0)."""
    nu = C / (np.asarray(lam_nm, dtype=np.float64) * 1e-7)
    w = np.zeros_like(nu)
    idx = np.flatnonzero(np.asarray(tag) == line)
    idx = idx[np.argsort(nu[idx])]
    for a, b in zip(idx[:-1], idx[1:]):
        h = nu[b] - nu[a]
        w[a] += 0.5 * h
        w[b] += 0.5 * h
    return w


def profiles(atom, lam_nm, tag, T):
    """Renormalised Doppler profiles phi[l][cell] (0 for continuum points / empty cells)."""
    lam_nm = np.asarray(lam_nm, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    nu = C / (lam_nm * 1e-7)
    phi = np.zeros((lam_nm.size,) + T.shape)
    for li, (lo, up, A, lam0) in enumerate(atom["lines"]):
        nu0 = C / (lam0 * 1e-7)
        with np.errstate(invalid="ignore", divide="ignore"):
            dnu = nu0 / C * np.sqrt(2.0 * K_B * T / (atom["mass_amu"] * AMU))
        sel = np.flatnonzero(np.asarray(tag) == li)
        w = frequency_weights(lam_nm, tag, li)
        raw = np.zeros((sel.size,) + T.shape)
        for q, k in enumerate(sel):
            with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
                raw[q] = np.where(T > 0, np.exp(-((nu[k] - nu0) / dnu) ** 2) / (np.sqrt(np.pi) * dnu), 0.0)
        norm = np.tensordot(w[sel], raw, axes=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            raw = np.where(norm > 0, raw / norm, 0.0)
        phi[sel] = raw
    return phi


def lte_populations(atom, T, nh):
    """Boltzmann populations [n_level][cell] summing to n_H (0 where T <= 0)."""
    T = np.asarray(T, dtype=np.float64)
    nh = np.asarray(nh, dtype=np.float64)
    E = np.asarray(atom["energy_ev"]) * EV
    g = np.asarray(atom["g"], dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        w = g[:, None] * np.exp(-E[:, None] / (K_B * T.reshape(-1)[None, :]))
        n = w / w.sum(axis=0) * nh.reshape(-1)[None, :]
    n = np.where(T.reshape(-1)[None, :] > 0, n, 0.0)
    return n.reshape((len(g),) + T.shape)


def eta_chi(atom, lam_nm, tag, T, ne, pops, cell_cm):
    """Per-cell float64 eta, chi ``[n_lambda][...]`` of the lines plus the grey background."""
    lam_nm = np.asarray(lam_nm, dtype=np.float64)
    nu = C / (lam_nm * 1e-7)
    T = np.asarray(T, dtype=np.float64)
    ne = np.asarray(ne, dtype=np.float64)
    phi = profiles(atom, lam_nm, tag, T)
    bs = einstein_b(atom)
    eta = np.zeros((lam_nm.size,) + T.shape)
    chi = np.zeros((lam_nm.size,) + T.shape)
    for k in range(lam_nm.size):
        chi_c = SIGMA_C * ne
        eta_c = chi_c * planck_nu(nu[k], T)
        e, x = eta_c, chi_c
        li = int(tag[k])
        if li >= 0:
            lo, up, A, _ = atom["lines"][li]
            b_ul, b_lu = bs[li]
            f = H * nu[k] / (4.0 * np.pi) * phi[k]
            e = e + f * pops[up] * A
            x = x + f * (pops[lo] * b_lu - pops[up] * b_ul)
        eta[k] = e * cell_cm
        chi[k] = x * cell_cm
    return eta, chi


def jbar(atom, lam_nm, tag, T, J):
    """Profile-weighted mean intensity per line ``[n_line][...]`` from J ``[n_lambda][...]``."""
    phi = profiles(atom, lam_nm, tag, T)
    out = []
    for li in range(len(atom["lines"])):
        w = frequency_weights(lam_nm, tag, li)
        out.append(np.tensordot(w, phi * np.asarray(J, dtype=np.float64), axes=1))
    return np.array(out)


def rate_matrix(atom, T, ne, Jbar):
    """P[i][j][...] = radiative + collisional rate from level i to level j."""
    T = np.asarray(T, dtype=np.float64)
    ne = np.asarray(ne, dtype=np.float64)
    nl = len(atom["g"])
    g = np.asarray(atom["g"], dtype=np.float64)
    E = np.asarray(atom["energy_ev"]) * EV
    P = np.zeros((nl, nl) + T.shape)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for (i, j), ups in atom["upsilon"].items():
            dE = E[j] - E[i]
            cij = ne * COLL / (g[i] * np.sqrt(T)) * ups * np.exp(-dE / (K_B * T))
            cji = ne * COLL / (g[j] * np.sqrt(T)) * ups
            P[i, j] += np.where(T > 0, cij, 0.0)
            P[j, i] += np.where(T > 0, cji, 0.0)
    for li, ((lo, up, A, _), (b_ul, b_lu)) in enumerate(zip(atom["lines"], einstein_b(atom))):
        P[lo, up] += b_lu * Jbar[li]
        P[up, lo] += A + b_ul * Jbar[li]
    return P


def se_solve(atom, T, ne, nh, Jbar):
    """Statistical-equilibrium populations ``[n_level][...]`` (0 where T <= 0)."""
    T = np.asarray(T, dtype=np.float64)
    shape = T.shape
    P = rate_matrix(atom, T, ne, Jbar).reshape(len(atom["g"]), len(atom["g"]), -1)
    nl = P.shape[0]
    M = np.zeros((P.shape[2], nl, nl))
    for i in range(nl):
        for j in range(nl):
            if i != j:
                M[:, i, j] += P[j, i]     # inflow j -> i
                M[:, i, i] -= P[i, j]     # outflow i -> j
    rhs = np.zeros((P.shape[2], nl))
    M[:, 0, :] = 1.0
    rhs[:, 0] = np.asarray(nh, dtype=np.float64).reshape(-1)
    live = T.reshape(-1) > 0
    n = np.zeros((P.shape[2], nl))
    if live.any():
        n[live] = np.linalg.solve(M[live], rhs[live][..., None])[..., 0]
    return n.T.reshape((nl,) + shape)
