"""Pins of the radiance-cascade oracle against facts that do not come from it:
the one-cascade limit (the separately pinned long-characteristics oracle),
closed forms in uniform media, exact reproduction of linear fields by the
bilinear merge, the direction nesting of branching factor 2, and an independent
recursive brute force on a tiny grid.
"""

import math

import numpy as np
import pytest

import synth
from oracle import lc, rc


def test_geometry_of_branching_factor_2():
    # Section 4.1: interval ends 1.5, 6, 24, ... voxels; 4x directions, 2x spacing
    g = rc.geometry(6, 4)
    assert [x[0] for x in g] == [1, 2, 4, 8, 16, 32]
    assert [x[1] for x in g] == [4, 16, 64, 256, 1024, 4096]
    assert [x[3] for x in g] == [1.5, 6.0, 24.0, 96.0, 384.0, 1536.0]
    assert [x[2] for x in g] == [0.0, 1.5, 6.0, 24.0, 96.0, 384.0]
    # every cascade holds the same number of (probe, direction) pairs on a 64^2 grid
    assert len({(64 // s) ** 2 * n for s, n, _, _ in g}) == 1


def test_child_directions_split_their_parent():
    dirs = synth.rc_directions(4, 4)
    for i in range(3):
        th = np.arctan2(dirs[i][:, 1].astype(np.float64), dirs[i][:, 0].astype(np.float64)) % (2 * np.pi)
        thc = np.arctan2(dirs[i + 1][:, 1].astype(np.float64), dirs[i + 1][:, 0].astype(np.float64)) % (2 * np.pi)
        thc = thc.reshape(-1, 4)
        # the four children are spaced 2 pi / N_{i+1} apart, centred on the parent
        np.testing.assert_allclose(np.unwrap(thc, axis=1).mean(axis=1) % (2 * np.pi), th, atol=1e-6)
        np.testing.assert_allclose(np.diff(np.unwrap(thc, axis=1), axis=1), 2 * np.pi / thc.size, atol=1e-6)
    np.testing.assert_array_equal(dirs[0], synth.directions(4)[0])


def test_one_cascade_is_long_characteristics():
    m = synth.random_medium(20, 14, 3, seed=synth.SEED_BASE + 300)
    eta, chi = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    n0 = 16
    dirs = synth.rc_directions(n0, 1)
    J = rc.rc_solve((eta, chi), 1, n0, dirs, t0=1e6, i_bc=0.4)
    Jlc = lc.formal_solve(eta, chi, dirs[0], np.full(n0, 1.0 / n0), i_bc=0.4)
    np.testing.assert_allclose(J, Jlc, rtol=1e-13, atol=0)


def test_uniform_medium_with_source_boundary_gives_source_everywhere():
    # I + T S = S(1 - T) + T S = S whatever the path lengths and weights
    chi = np.full((1, 32, 32), 0.3)
    eta = 1.7 * chi
    dirs = synth.rc_directions(4, 4)
    J = rc.rc_solve((eta, chi), 4, 4, dirs, i_bc=1.7)
    np.testing.assert_allclose(J, 1.7, rtol=1e-14)


def test_uniform_medium_interior_closed_form():
    # Far enough from the boundary no interval of any cascade leaves the grid and
    # every interpolation stencil sees equal values: the cascades compose exactly
    # to S (1 - exp(-chi t_end)) with t_end the end of the top interval (24).
    n = 128
    chi0, S = 0.05, 2.0
    eta = np.full((1, n, n), chi0 * S)
    chi = np.full((1, n, n), chi0)
    dirs = synth.rc_directions(4, 3)
    J = rc.rc_solve((eta, chi), 3, 4, dirs, i_bc=0.0).reshape(n, n)
    ref = S * (1 - math.exp(-chi0 * 24.0))
    interior = J[40:88, 40:88]
    np.testing.assert_allclose(interior, ref, rtol=1e-12)
    assert abs(J[0, 0] - ref) > 1e-3     # near the corner rays leave the grid early


def test_bilinear_merge_reproduces_linear_fields():
    # an upper field linear in the probe coordinates (same in every child
    # direction) is reproduced exactly at interior finer probes
    qz, qx, n_dir = 8, 12, 3
    zc = 2 * (np.arange(qz) + 0.5)           # coarse probe coordinates, fine spacing 1
    xc = 2 * (np.arange(qx) + 0.5)
    f = lambda z, x: 0.3 + 0.7 * z - 1.1 * x
    up = np.broadcast_to(f(zc[:, None], xc[None, :])[None, :, :, None], (4 * n_dir, qz, qx, 1)).copy()
    R = rc.upper_radiance(up, n_dir, 2 * qz, 2 * qx)
    zf = np.arange(2 * qz) + 0.5
    xf = np.arange(2 * qx) + 0.5
    ref = f(zf[:, None], xf[None, :])
    np.testing.assert_allclose(R[:, 1:-1, 1:-1, 0], np.broadcast_to(ref[1:-1, 1:-1], (n_dir, 2 * qz - 2, 2 * qx - 2)),
                               rtol=1e-14, atol=1e-13)
    # at the edge the stencil clamps: the first probe takes the first coarse value
    np.testing.assert_allclose(R[0, 0, 0, 0], f(zc[0], xc[0]), rtol=1e-14)


def _brute_force_J(eta, chi, C, n0, dirs, i_bc):
    """Independent evaluation: each merged radiance is computed by recursion on
    demand, straight from the definition, with per-probe, per-ray plane walks."""
    L, nz, nx = eta.shape
    geo = rc.geometry(C, n0)
    memo = {}

    def walk(i, pz, px, k):
        s, _, t_s, t_e = geo[i]
        ox, oz = s * (px + 0.5), s * (pz + 0.5)
        dx, dz = float(dirs[i][k, 0]), float(dirs[i][k, 1])
        # exit parameter
        tx = (nx - ox) / dx if dx > 0 else (-ox / dx if dx < 0 else math.inf)
        tz = (nz - oz) / dz if dz > 0 else (-oz / dz if dz < 0 else math.inf)
        t_exit = min(tx, tz)
        # fine sub-steps: cell of each sub-step midpoint (brute force), from the far end
        tb = min(t_e, t_exit)
        I = np.zeros(L)
        T = np.ones(L)
        if tb > t_s:
            n_sub = max(1, int(math.ceil((tb - t_s) / 2e-3)))
            h = (tb - t_s) / n_sub
            for q in range(n_sub - 1, -1, -1):
                tm = t_s + (q + 0.5) * h
                ci = min(max(int(math.floor(ox + tm * dx)), 0), nx - 1)
                cj = min(max(int(math.floor(oz + tm * dz)), 0), nz - 1)
                x, e = chi[:, cj, ci], eta[:, cj, ci]
                att = np.exp(-x * h)
                src = np.where(x > 0, e / np.where(x > 0, x, 1) * (1 - att), e * h)
                I = I * att + src
                T = T * att
        return I, T, t_exit <= t_e

    def radiance(i, pz, px, k):
        key = (i, pz, px, k)
        if key in memo:
            return memo[key]
        I, T, left = walk(i, pz, px, k)
        if left or i == C - 1:
            R = np.full(L, i_bc)
        else:
            qz, qx = nz // 2 ** (i + 1), nx // 2 ** (i + 1)
            uz, ux = (pz + 0.5) / 2 - 0.5, (px + 0.5) / 2 - 0.5
            z0, x0 = math.floor(uz), math.floor(ux)
            fz, fx = uz - z0, ux - x0
            R = np.zeros(L)
            for (zz, wz) in ((z0, 1 - fz), (z0 + 1, fz)):
                for (xx, wx) in ((x0, 1 - fx), (x0 + 1, fx)):
                    zq, xq = min(max(zz, 0), qz - 1), min(max(xx, 0), qx - 1)
                    R += wz * wx * sum(radiance(i + 1, zq, xq, 4 * k + c) for c in range(4)) / 4
        out = I + T * R
        memo[key] = out
        return out

    J = np.zeros((L, nz * nx))
    for pz in range(nz):
        for px in range(nx):
            J[:, pz * nx + px] = sum(radiance(0, pz, px, k) for k in range(n0)) / n0
    return J


def test_brute_force_recursion_on_a_tiny_grid():
    m = synth.random_medium(8, 8, 2, seed=synth.SEED_BASE + 301, log_chi_range=(-2.0, 0.5))
    eta, chi = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    dirs = synth.rc_directions(4, 3)
    J = rc.rc_solve((eta, chi), 3, 4, dirs, i_bc=0.25)
    Jb = _brute_force_J(eta, chi, 3, 4, dirs, 0.25)
    # the brute force sub-steps at 2e-3 voxel (observed agreement 2.3e-4)
    np.testing.assert_allclose(J, Jb, rtol=1e-3, atol=0)
