"""Pins of the statistical-equilibrium oracle against physics that does not come from
the oracle: Stefan-Boltzmann, the Rayleigh-Jeans and Wien limits, Kirchhoff's law
(S = B in LTE), detailed balance (J = B gives Boltzmann populations), conservation,
and the profile normalisation."""

import math

import numpy as np

import synth
from synth.atom import three_level_atom, line_wavelength_grid
from oracle import atom as oa


def consistent_atom():
    """The synthetic atom with rest wavelengths set exactly from the level energies,
    so that LTE identities hold to rounding."""
    a = three_level_atom()
    E = np.asarray(a["energy_ev"]) * oa.EV
    a = dict(a)
    a["lines"] = [(lo, up, A, oa.H * oa.C / (E[up] - E[lo]) * 1e7) for (lo, up, A, _) in a["lines"]]
    return a


def test_planck_integral_and_limits():
    T = 7000.0
    nu = np.geomspace(1e11, 1e17, 200001)
    B = oa.planck_nu(nu, T)
    integral = np.trapezoid(B, nu)
    sigma_sb = 2 * math.pi ** 5 * oa.K_B ** 4 / (15 * oa.C ** 2 * oa.H ** 3)
    assert abs(integral / (sigma_sb * T ** 4 / math.pi) - 1) < 1e-5
    nu_rj = 1e9  # h nu / k T ~ 7e-6
    assert abs(oa.planck_nu(nu_rj, T) / (2 * nu_rj ** 2 * oa.K_B * T / oa.C ** 2) - 1) < 1e-5
    nu_w = 5e15  # h nu / k T ~ 34
    wien = 2 * oa.H * nu_w ** 3 / oa.C ** 2 * math.exp(-oa.H * nu_w / (oa.K_B * T))
    assert abs(oa.planck_nu(nu_w, T) / wien - 1) < 1e-13


def test_profile_quadrature_is_normalised():
    a = three_level_atom()
    lam, tag = line_wavelength_grid(24, 8)
    T = np.array([5e3, 2e4, 9e4])
    phi = oa.profiles(a, lam, tag, T)
    for li in range(2):
        w = oa.frequency_weights(lam, tag, li)
        np.testing.assert_allclose(np.tensordot(w, phi, axes=1), 1.0, rtol=1e-13)
    assert (phi[tag == -1] == 0).all()


def test_kirchhoff_lte_source_function_is_planck():
    a = consistent_atom()
    lam, tag = line_wavelength_grid(16, 4)
    T = np.array([6e3, 1.5e4, 4e4])
    ne = np.array([1e11, 1e13, 1e15])
    nh = 10 * ne
    pops = oa.lte_populations(a, T, nh)
    eta, chi = oa.eta_chi(a, lam, tag, T, np.zeros_like(ne), pops, 1e6)  # lines only
    for k in np.flatnonzero(tag >= 0):
        lo, up, A, lam0 = a["lines"][tag[k]]
        nu0 = oa.C / (lam0 * 1e-7)
        np.testing.assert_allclose(eta[k] / chi[k], oa.planck_nu(nu0, T), rtol=1e-12)


def test_detailed_balance_and_lte_recovery():
    a = consistent_atom()
    T = np.array([5e3, 1e4, 3e4, 1e5])
    ne = np.array([1e9, 1e12, 1e15, 1e17])
    nh = 10 * ne
    P = oa.rate_matrix(a, T, ne, np.zeros((2, 4)))
    E = np.asarray(a["energy_ev"]) * oa.EV
    g = np.asarray(a["g"])
    for (i, j) in a["upsilon"]:
        ratio = P[j, i] / P[i, j] if (i, j) not in [(0, 1), (1, 2)] else None
        if ratio is not None:
            np.testing.assert_allclose(ratio, g[i] / g[j] * np.exp((E[j] - E[i]) / (oa.K_B * T)), rtol=1e-12)
    # J = B(nu0) in every line -> Boltzmann populations
    Jbar = np.array([oa.planck_nu(oa.C / (lam0 * 1e-7), T) for (_, _, _, lam0) in a["lines"]])
    n = oa.se_solve(a, T, ne, nh, Jbar)
    np.testing.assert_allclose(n, oa.lte_populations(a, T, nh), rtol=1e-9)
    np.testing.assert_allclose(n.sum(axis=0), nh, rtol=1e-13)


def test_two_level_ratio_when_third_level_is_decoupled():
    # With the third level reachable only through a vanishing collision strength the
    # 1-2 ratio is the two-level closed form n2/n1 = (B12 J + C12) / (A21 + B21 J + C21).
    a = consistent_atom()
    a["lines"] = a["lines"][:1]
    a["upsilon"] = {(0, 1): 0.5, (0, 2): 1e-30, (1, 2): 1e-30}
    T = np.array([8000.0])
    ne = np.array([1e13])
    J = np.array([[3e-6]])
    n = oa.se_solve(a, T, ne, 10 * ne, J)
    (b21, b12), = oa.einstein_b(a)
    A = a["lines"][0][2]
    E = np.asarray(a["energy_ev"]) * oa.EV
    c12 = ne * oa.COLL / (2 * math.sqrt(T[0])) * 0.5 * math.exp(-(E[1] - E[0]) / (oa.K_B * T[0]))
    c21 = ne * oa.COLL / (8 * math.sqrt(T[0])) * 0.5
    ref = (b12 * J[0] + c12) / (A + b21 * J[0] + c21)
    assert abs(n[1, 0] / n[0, 0] / ref[0] - 1) < 1e-9


def test_empty_cells_have_no_populations():
    a = three_level_atom()
    m = synth.atom.populations_atmosphere(64, 48, seed=7)
    pops = oa.lte_populations(a, m["temperature"], m["nh"])
    assert (pops[:, m["temperature"] == 0] == 0).all()
    live = m["temperature"] > 0
    np.testing.assert_allclose(pops.sum(axis=0)[live], m["nh"][live].astype(np.float64), rtol=1e-12)
