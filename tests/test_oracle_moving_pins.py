"""Pins of the moving-medium oracles (oracle/cav.py, oracle/velinterp.py) against
facts the paper and the mathematics fix, independent of the oracles' own code:

* Section 3.2's Doppler relation phi_l(lambda, w) = phi_l(lambda + (v . w / c) lambda0):
  a medium moving with uniform v seen along w has, at wavelength offset dv, the
  rest-frame profile at dv + v . w (with the lambda0 / lambda factors frozen, c -> inf);
* the static limit is the normalised Voigt profile of scipy's ``voigt_profile``
  (Gaussian of standard deviation v_th / sqrt 2 convolved with a Lorentzian of
  half width a v_th), checked cell by cell;
* Section 3.2.1's scalings at one wavelength: eta*, chi* times lambda0 / lambda
  and the damping times (lambda / lambda0)^2;
* the closest-to-core shift of the CaV level test, by hand, for |dv| < |v| and
  |dv| > |v|;
* Section 3.1's velocity grids: samples at v_s = -V + 2 V s / (n - 1) with V the
  largest speed of the voxel's MIP-0 cells, each the mean over those cells of
  the cell's value at projected velocity v_s; linear interpolation reproduces a
  field linear in the projected velocity exactly, clamps outside [-V, V], and a
  voxel at rest (V = 0) has a constant grid;
* the direction convention (the intensity of a ray traced toward +d propagates
  along w = -d) in a whole CaV formal solve through a uniformly moving slab.
A planted sign flip of v . w, a dropped lambda0 / lambda, a wrong shift or a wrong
V per voxel fails at least one of these.
"""

import math

import numpy as np
import pytest
from scipy.special import erfcx, voigt_profile

from oracle import cav, lc, velinterp as ov

C_INF = 1e30


def cells(n=(2, 4), seed=3, vmax=40.0):
    """Parameter fields P [8][nz][nx] of a small medium with varied values."""
    rng = np.random.default_rng(seed)
    nz, nx = n
    m = {
        "eta_star": rng.uniform(0.5, 2.0, n), "chi_star": rng.uniform(1.0, 5.0, n),
        "damping": 10.0 ** rng.uniform(-3, -1, n), "vth": rng.uniform(5.0, 10.0, n),
        "vx": rng.uniform(-vmax, vmax, n), "vz": rng.uniform(-vmax, vmax, n),
        "eta_c": rng.uniform(0.0, 0.1, n), "chi_c": rng.uniform(0.01, 0.1, n),
    }
    return m, cav.param_arrays(m)


def phi(dv, vth, a):
    return voigt_profile(dv, vth / math.sqrt(2.0), a * vth)


def test_static_limit_is_the_normalised_voigt_profile():
    m, P = cells()
    P[4] = P[5] = 0.0
    dv = np.array([-17.0, -3.5, 0.0, 2.25, 40.0])
    eta, chi = cav.eta_chi(P, dv, 0.3, -0.7, C_INF)
    for k in range(dv.size):
        ph = phi(dv[k], m["vth"], m["damping"])
        np.testing.assert_allclose(eta[k], m["eta_star"] * ph + m["eta_c"], rtol=1e-12)
        np.testing.assert_allclose(chi[k], m["chi_star"] * ph + m["chi_c"], rtol=1e-12)


def test_uniform_velocity_is_a_doppler_shift_of_the_rest_profile():
    m, P = cells()
    vx, vz = 23.0, -11.0
    P[4], P[5] = vx, vz
    dv = np.linspace(-60, 60, 13)
    for wx, wz in ((1.0, 0.0), (0.0, -1.0), (0.6, 0.8), (-0.28, 0.96)):
        eta, chi = cav.eta_chi(P, dv, wx, wz, C_INF)
        shift = vx * wx + vz * wz                      # v . w in km/s
        for k in range(dv.size):
            ph = phi(dv[k] + shift, m["vth"], m["damping"])
            np.testing.assert_allclose(eta[k], m["eta_star"] * ph + m["eta_c"], rtol=1e-12)
            np.testing.assert_allclose(chi[k], m["chi_star"] * ph + m["chi_c"], rtol=1e-12)


def test_wavelength_scalings_at_one_wavelength():
    # c chosen so that lambda0 / lambda = 1 / (1 + dv / c) = 2/3 at dv = 50:
    # eta*, chi* scale by 2/3, the damping by (3/2)^2, the profile argument stays dv / v_th
    m, P = cells()
    P[4] = P[5] = 0.0
    c, dv = 100.0, np.array([50.0])
    s = 2.0 / 3.0
    eta, chi = cav.eta_chi(P, dv, 1.0, 0.0, c)
    ph = phi(50.0, m["vth"], m["damping"] / (s * s))
    np.testing.assert_allclose(eta[0], s * m["eta_star"] * ph + m["eta_c"], rtol=1e-12)
    np.testing.assert_allclose(chi[0], s * m["chi_star"] * ph + m["chi_c"], rtol=1e-12)


def test_closest_to_core_shift_by_hand():
    m, P = cells(n=(1, 2))
    P[4] = np.array([[3.0, 0.0]])      # speeds 5 and 13 km/s
    P[5] = np.array([[4.0, -13.0]])
    vth, a = m["vth"][0], m["damping"][0]
    for dv in (-20.0, -9.0, 0.0, 4.0, 5.0, 12.0, 31.0):
        eta, _ = cav.eta_chi(P, np.array([dv]), 0.0, 0.0, C_INF, closest_to_core=True)
        for c, speed in ((0, 5.0), (1, 13.0)):
            u = max(abs(dv) - speed, 0.0)      # |dv| < |v|: the line centre itself is reachable
            ref = m["eta_star"][0, c] * phi(u, vth[c], a[c]) + m["eta_c"][0, c]
            assert abs(eta[0, 0, c] - ref) <= 1e-12 * ref, (dv, c)
            if abs(dv) <= speed:   # at the line centre H(a, 0) = e^{a^2} erfc(a)
                assert abs(eta[0, 0, c] - (m["eta_star"][0, c] * erfcx(a[c]) / (math.sqrt(math.pi) * vth[c])
                                           + m["eta_c"][0, c])) <= 1e-12 * ref


def test_velocity_grid_samples_and_voxel_speed_by_hand():
    m, P = cells(n=(2, 2), seed=7)
    dv = np.array([-8.0, 0.0, 15.0])
    g = ov.velocity_grids(P, dv, C_INF, 1, n_vel=8, method="exact")
    speed = np.hypot(m["vx"], m["vz"])
    # MIP 0: each cell's own speed, samples at -V + 2 V s / 7, the cell's rest profile shifted
    np.testing.assert_allclose(g[0]["V"], speed, rtol=1e-15)
    for s in range(8):
        vs = -speed + 2.0 * speed * s / 7.0
        for k in range(dv.size):
            ph = phi(dv[k] + vs, m["vth"], m["damping"])
            np.testing.assert_allclose(g[0]["eta"][s, k], m["eta_star"] * ph + m["eta_c"], rtol=1e-12)
            np.testing.assert_allclose(g[0]["chi"][s, k], m["chi_star"] * ph + m["chi_c"], rtol=1e-12)
    # MIP 1: the 2x2 voxel's V is the largest of its four speeds; sample s is the mean of
    # the four cells' values at that one projected velocity; the mean velocity is the box mean
    V = speed.max()
    assert g[1]["V"].shape == (1, 1) and abs(g[1]["V"][0, 0] - V) <= 1e-14 * V
    assert abs(g[1]["vx"][0, 0] - m["vx"].mean()) < 1e-12 and abs(g[1]["vz"][0, 0] - m["vz"].mean()) < 1e-12
    for s in (0, 3, 7):
        vs = -V + 2.0 * V * s / 7.0
        ph = phi(dv[2] + vs, m["vth"], m["damping"])
        assert abs(g[1]["eta"][s, 2, 0, 0] - np.mean(m["eta_star"] * ph + m["eta_c"])) < 1e-12


def test_interpolation_is_exact_for_fields_linear_in_velocity():
    rng = np.random.default_rng(11)
    V = np.array([[0.0, 7.0, 30.0]])
    vx, vz = np.array([[5.0, 3.0, -20.0]]), np.array([[1.0, -6.0, 25.0]])
    alpha, beta = rng.uniform(1, 2, (2, 1, 3)), rng.uniform(-0.05, 0.05, (2, 1, 3))
    vs = np.stack([-V + 2 * V * s / 7.0 for s in range(8)])                  # [8][1][3]
    grid = {"V": V, "vx": vx, "vz": vz,
            "eta": (alpha[0][None, None] + beta[0][None, None] * vs[:, None]),   # [8][L=1][1][3]
            "chi": (alpha[1][None, None] + beta[1][None, None] * vs[:, None])}
    for wx, wz in ((1.0, 0.0), (0.0, 1.0), (0.6, -0.8), (-1.0, 0.0)):
        e, c = ov.interpolate(grid, wx, wz)
        proj = np.clip(vx * wx + vz * wz, -V, V)     # clamped to the grid's range
        np.testing.assert_allclose(e[0], alpha[0] + beta[0] * proj, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(c[0], alpha[1] + beta[1] * proj, rtol=1e-13, atol=1e-15)
    # the first voxel is at rest (V = 0): every direction returns its constant grid value
    e0 = [ov.interpolate(grid, wx, wz)[0][0, 0, 0] for wx, wz in ((1, 0), (0, 1), (-0.6, 0.8))]
    assert e0[0] == e0[1] == e0[2] == alpha[0][0, 0]


def test_voxel_at_rest_has_a_constant_grid():
    m, P = cells(n=(2, 2), seed=9)
    P[4] = P[5] = 0.0
    g = ov.velocity_grids(P, np.array([-5.0, 1.0]), C_INF, 1, n_vel=8)
    for lvl in g:
        assert np.all(lvl["V"] == 0.0)
        assert np.all(lvl["eta"] == lvl["eta"][:1]) and np.all(lvl["chi"] == lvl["chi"][:1])


@pytest.mark.usefixtures("oracle_lib")
def test_cav_solve_through_a_moving_slab_uses_propagation_direction():
    # a 16 x 16 uniform slab moving with v = (30, 0) km/s; the ray traced toward +x
    # carries light propagating along -x (w = -d), which sees the profile at dv - 30,
    # the ray traced toward -x the profile at dv + 30
    n = 16
    m = {"eta_star": np.full((n, n), 2.0), "chi_star": np.full((n, n), 0.5), "damping": np.full((n, n), 0.01),
         "vth": np.full((n, n), 6.0), "vx": np.full((n, n), 30.0), "vz": np.zeros((n, n)),
         "eta_c": np.full((n, n), 0.001), "chi_c": np.full((n, n), 0.002)}
    P = cav.param_arrays(m)
    dv = np.array([-30.0, 0.0, 30.0])
    dirs = np.array([[1.0, 0.0], [-1.0, 0.0]])
    probes = np.array([5 * n + 3, 8 * n + 12], dtype=np.int32)
    lev = np.zeros((1, 1, 1), dtype=np.int32)
    _, I = cav.formal_solve([P], lev, 16, 8, dv, C_INF, dirs, [0.5, 0.5], probes, method="exact",
                            want_intensity=True)
    for k, shift in ((0, -30.0), (1, 30.0)):
        ph = phi(dv + shift, 6.0, 0.01)
        eta = (2.0 * ph + 0.001)[:, None, None] * np.ones((1, n, n))
        chi = (0.5 * ph + 0.002)[:, None, None] * np.ones((1, n, n))
        _, Ir = lc.formal_solve(eta, chi, dirs[k:k + 1], [1.0], probes=probes, want_intensity=True)
        np.testing.assert_allclose(I[:, k, :], Ir[:, 0, :], rtol=1e-12)
        # and the closed form of a uniform slab: I = S (1 - e^{-chi l}), l = distance to the edge
        ell = (n - 3 - 0.5, n - 12 - 0.5) if k == 0 else (3 + 0.5, 12 + 0.5)
        for p, l_ in enumerate(ell):
            np.testing.assert_allclose(I[:, k, p], eta[:, 0, 0] / chi[:, 0, 0] * -np.expm1(-chi[:, 0, 0] * l_),
                                       rtol=1e-12)
