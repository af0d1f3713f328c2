"""Pins of the MALI oracle (oracle/mali.py) against facts that do not use it:

* the diagonal operator: on a one-cell grid the long-characteristics oracle's J
  is exactly Lambda* S (the ray leaves the cell after l_k), for any opacity;
* thin limit: with vanishing opacity Lambda* -> 0, Psibar -> 0 and Jbar_eff ->
  Jbar, so one MALI update is one Lambda-iteration update;
* fixed point: at the exact statistical-equilibrium populations n* of an
  isolated cell (found here by a root finder on the exact equations
  n = SE(Jbar(n)) with J = Lambda*[S(n)]), the preconditioned rates reproduce
  the exact net rates and M(n*) = n*; at any other n, M(n) != n;
* convergence: a two-level atom in an isothermal slab converges monotonically
  to the populations the (slow) Lambda iteration approaches, in far fewer
  iterations; on the population workload's 48 x 48 instance with the MALI
  wavelength grid the iteration reaches a largest relative change < 1e-3.
A dropped chi_line / chi factor, a sign flip in Jbar_eff or the wrong own-cell
length breaks the fixed point or the one-cell identity.
"""

import numpy as np
import pytest
from scipy.optimize import root

import synth
from oracle import atom as oa, lc, mali, mips as omips
from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom

pytestmark = pytest.mark.usefixtures("oracle_lib")


def two_level():
    a = three_level_atom()
    return {"energy_ev": a["energy_ev"][:2], "g": a["g"][:2], "lines": [a["lines"][0]], "upsilon": {(0, 1): 0.5},
            "mass_amu": a["mass_amu"]}


def one_cell_J(eta, chi, dirs, w):
    return lc.formal_solve(eta.reshape(-1, 1, 1), chi.reshape(-1, 1, 1), dirs, w, probes=np.array([0], np.int32))


def test_lambda_star_is_the_one_cell_solution():
    dirs, w = synth.directions(24)
    chi = np.array([1e-6, 0.01, 0.3, 2.0, 40.0])
    S = np.array([1.0, 2.0, 0.5, 3.0, 1.5])
    J = one_cell_J(chi * S, chi, dirs, w)[:, 0]
    np.testing.assert_allclose(J, mali.lambda_star(chi, dirs, w) * S, rtol=1e-12)
    # and the own-cell length by hand for a diagonal and an axis ray
    np.testing.assert_allclose(mali.own_cell_lengths([[1.0, 0.0], [0.6, 0.8], [-2 ** -0.5, 2 ** -0.5]]),
                               [0.5, 0.625, 2 ** -0.5], rtol=1e-15)


def test_thin_limit_is_one_lambda_step():
    atom = three_level_atom()
    lam, tag = line_wavelength_grid(t_ref=1e5)
    dirs, w = synth.directions(16)
    T, ne = np.array([8e3, 2e4, 6e4]), np.array([1e2, 1e3, 1e2])     # tenuous: every cell optically thin
    nh = 10 * ne
    pops = oa.lte_populations(atom, T, nh) * np.array([[1.1], [0.7], [1.3]])
    rng = np.random.default_rng(2)
    J = rng.uniform(0.5, 2.0, (lam.size, 3)) * oa.planck_nu(oa.C / (lam[:, None] * 1e-7), T[None])
    new = mali.mali_step(atom, lam, tag, T, ne, nh, 1e-3, pops, J, dirs, w)
    ref = oa.se_solve(atom, T, ne, nh, oa.jbar(atom, lam, tag, T, J))
    np.testing.assert_allclose(new, ref, rtol=1e-9)


@pytest.mark.parametrize("T,ne", [(8e3, 1e12), (3e4, 3e10), (6e4, 5e9)])
def test_exact_populations_are_the_fixed_point(T, ne):
    atom = three_level_atom()
    lam, tag = line_wavelength_grid(t_ref=1e5)
    dirs, w = synth.directions(16)
    Ta, nea, nha = np.array([T]), np.array([ne]), np.array([10 * ne])
    cell = 1e6

    def exact_map(n):
        eta, chi = oa.eta_chi(atom, lam, tag, Ta, nea, n.reshape(3, 1), cell)
        J = one_cell_J(eta, chi, dirs, w)
        return oa.se_solve(atom, Ta, nea, nha, oa.jbar(atom, lam, tag, Ta, J)).reshape(-1)

    n0 = oa.lte_populations(atom, Ta, nha).reshape(-1)
    sol = root(lambda x: exact_map(x * n0) / n0 - x, np.ones(3), method="lm", tol=1e-14)
    nstar = (sol.x * n0).reshape(3, 1)
    assert np.abs(exact_map(nstar.reshape(-1)) - nstar.reshape(-1)).max() < 1e-10 * nstar.max()

    def M(n):
        eta, chi = oa.eta_chi(atom, lam, tag, Ta, nea, n, cell)
        return mali.mali_step(atom, lam, tag, Ta, nea, nha, cell, n, one_cell_J(eta, chi, dirs, w), dirs, w)
    np.testing.assert_allclose(M(nstar), nstar, rtol=1e-8)
    off = nstar * np.array([[1.05], [0.97], [0.9]])
    assert np.abs(M(off) / off - 1).max() > 1e-4


def slab_solver(N, dirs, w):
    def solve_J(eta, chi):
        return lc.formal_solve(eta.reshape(-1, N, N), chi.reshape(-1, N, N), dirs, w)
    return solve_J


def test_isothermal_slab_two_level_converges_monotonically():
    atom = two_level()
    lam, tag = line_wavelength_grid(t_ref=1e5)
    sel = tag == 0
    lam, tag = lam[sel], tag[sel]
    N = 16
    dirs, w = synth.directions(8)
    T = np.full((N, N), 8e3)
    ne = np.full((N, N), 1e10)
    nh = 10 * ne
    solve_J = slab_solver(N, dirs, w)
    pm, nm, hm = mali.iterate(atom, lam, tag, T, ne, nh, 1e6, solve_J, dirs, w, tol=1e-6, max_iter=60)
    assert nm < 60 and all(b < a for a, b in zip(hm[1:], hm[2:])), hm
    # the Lambda iteration from LTE creeps toward the same populations
    p = oa.lte_populations(atom, T.reshape(-1), nh.reshape(-1))
    gaps = []
    for _ in range(nm):
        eta, chi = oa.eta_chi(atom, lam, tag, T.reshape(-1), ne.reshape(-1), p, 1e6)
        J = solve_J(eta, chi)
        p = oa.se_solve(atom, T.reshape(-1), ne.reshape(-1), nh.reshape(-1), oa.jbar(atom, lam, tag, T.reshape(-1), J))
        gaps.append(np.abs(p / pm - 1).max())
    assert gaps[-1] < gaps[0] and gaps[-1] > 100 * hm[-1]   # same direction, far slower


def test_population_workload_converges():
    atom = three_level_atom()
    lam, tag = line_wavelength_grid(t_ref=1e5)
    N = 48
    m = populations_atmosphere(N, N, seed=synth.SEED_BASE + 4)
    T, ne, nh = (m[k].astype(np.float64) for k in ("temperature", "ne", "nh"))
    dirs, w = synth.directions(16)

    def solve_J(eta, chi):
        e, c = eta.reshape(-1, N, N), chi.reshape(-1, N, N)
        probes = omips.probes_of_blocks(omips.block_empty(e, c, 16), 16)
        J = np.zeros((lam.size, N * N))
        J[:, probes] = lc.formal_solve(e, c, dirs, w, probes=probes)
        return J
    p, n, h = mali.iterate(atom, lam, tag, T, ne, nh, m["cell_cm"], solve_J, dirs, w, tol=1e-3, max_iter=150)
    assert h[-1] < 1e-3 and n < 150, (n, h[-5:])
    live = T.reshape(-1) > 0
    assert np.all(p[:, live] > 0) and np.allclose(p[:, live].sum(0), nh.reshape(-1)[live], rtol=1e-10)
