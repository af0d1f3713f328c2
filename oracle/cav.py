"""Float64 oracle of the "Core and Voigt" (CaV) treatment of a moving medium (Section 3.2).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

Model (one line plus an isotropic background, velocities and wavelengths in km/s):
  propagation direction w = -d for a ray traced toward +d from the probe;
  u = dv + v . w            (Section 3.2: phi_l(lambda, w) = varphi_l(lambda + (v.w/c) lambda0))
  s = lambda0 / lambda = 1 / (1 + dv / c)
  eta = eta* s phi + eta_c,  chi = chi* s phi + chi_c,          (eta*(lambda) = (lambda0/lambda) eta*(lambda0))
  phi = H(a / s^2, u / v_th) / (sqrt(pi) v_th)                  (a(lambda) = (lambda/lambda0)^2 a(lambda0))
with H the Voigt function: the exact Faddeeva value (method "exact", the accuracy reference), or
HUM1WEI24 (the form the method evaluates) for parity with the GPU.

Acceleration (restated from Section 3.2 and Section 2.2):
  * MIP chains of eta*, chi*, a, 1/v_th, v_x, v_z, eta_c, chi_c (box filter);
  * the level of a block per wavelength batch from Eq. IoD applied to eta and chi
    evaluated, per voxel, at the Doppler shift closest to the line core that the
    voxel's speed allows (|u| = max(0, |dv| - |v|)), with the always-average rule;
  * along a ray, a block is sampled at its level (optionally distance limited);
    every MIP-0 cell of a voxel carries the voxel's parameters, so the plain
    solver over those per-cell values is the accelerated result.
"""

from __future__ import annotations

import numpy as np

from . import lc, mips as omips
from .voigt import voigt_h

PARAMS = ("eta_star", "chi_star", "damping", "inv_vth", "vx", "vz", "eta_c", "chi_c")


def param_arrays(m):
    """The 8 per-cell parameters as float64 [8][nz][nx] (1/v_th where v_th > 0, else 0)."""
    vth = np.asarray(m["vth"], dtype=np.float64)
    inv = np.where(vth > 0, 1.0 / np.where(vth > 0, vth, 1.0), 0.0)
    vals = {"inv_vth": inv}
    for k in ("eta_star", "chi_star", "damping", "vx", "vz", "eta_c", "chi_c"):
        vals[k] = np.asarray(m[k], dtype=np.float64)
    return np.stack([vals[k] for k in PARAMS])


def eta_chi(P, dv, wx, wz, c_kms, method="exact", closest_to_core=False, profile=None):
    """eta, chi [L][...] from parameters P [8][...] for propagation direction (wx, wz).

    With ``closest_to_core`` the projected velocity is replaced by the shift within
    [-|v|, |v|] closest to line centre (direction-free worst case of Section 3.2).
    ``profile(a, x, u)``, if given, replaces H(a, x - u) (x = dv / v_th, u = -(v.w) / v_th)."""
    es, cs, a, inv, vx, vz, ec, cc = P
    dv = np.asarray(dv, dtype=np.float64)
    L = dv.size
    eta = np.empty((L,) + es.shape)
    chi = np.empty((L,) + es.shape)
    speed = np.sqrt(vx * vx + vz * vz)
    for k in range(L):
        s = 1.0 / (1.0 + dv[k] / c_kms)
        if closest_to_core:
            u = np.maximum(np.abs(dv[k]) - speed, 0.0)
        else:
            u = dv[k] + vx * wx + vz * wz
        if profile is not None and not closest_to_core:
            H = profile(a / (s * s), dv[k] * inv, -(vx * wx + vz * wz) * inv)
        else:
            H = voigt_h(a / (s * s), u * inv, method=method)
        phi = H * inv / np.sqrt(np.pi)
        eta[k] = es * s * phi + ec
        chi[k] = cs * s * phi + cc
    return eta, chi


def param_chain(P0, max_mip):
    """Box-filter MIP chain of the parameters: list of [8][nz>>m][nx>>m]."""
    chain = [P0]
    for _ in range(max_mip):
        p = chain[-1]
        n, Z, X = p.shape
        chain.append(p.reshape(n, Z // 2, 2, X // 2, 2).mean(axis=(2, 4)))
    return chain


def test_directions(n_test_dirs):
    """The K in-plane propagation directions of the directional level test."""
    th = 2.0 * np.pi * np.arange(n_test_dirs) / max(n_test_dirs, 1)
    return list(zip(np.cos(th), np.sin(th)))


def block_levels(chain, dv, c_kms, empty, block, lambda_batch, thr_eta, thr_chi, chi_ds_min=0.25,
                 method="hum1wei24", stats=False, n_test_dirs=0):
    """Per-batch block levels from the closest-to-core IoD test over the chain's children.

    With ``n_test_dirs`` = K > 0 (a reading of the "worst-case gradients" the test
    is meant to bound) a group must also pass the same test on its children
    evaluated as a ray propagating along each w_k = (cos 2 pi k / K, sin 2 pi k / K)
    samples them: u = dv + v_child . w_k.  ``stats``: per level a dict of the
    closest-to-core test's quantities; with K > 0 a list of such per-level lists,
    one per evaluation (closest-to-core first, then the K directions)."""
    max_mip = len(chain) - 1
    passes = []
    st = [[] for _ in range(1 + n_test_dirs)]
    for m in range(1, max_mip + 1):
        ds = float(2 ** m)
        evals = [eta_chi(chain[m - 1], dv, 0.0, 0.0, c_kms, method=method, closest_to_core=True)]
        evals += [eta_chi(chain[m - 1], dv, wx, wz, c_kms, method=method) for wx, wz in test_directions(n_test_dirs)]
        ok = None
        for q, (e, x) in enumerate(evals):
            ge, gx = omips._groups(e), omips._groups(x)
            _, iod_e = omips._reduce(ge, ds, "linear")
            _, iod_c = omips._reduce(gx, ds, "linear")
            kds = gx.max(-1) * ds
            p = ((iod_e < thr_eta) & (iod_c < thr_chi)) | (kds < chi_ds_min)
            ok = p if ok is None else ok & p
            st[q].append({"iod_eta": iod_e, "iod_chi": iod_c, "chi_ds": kds})
        passes.append(ok)
    lev = omips.block_levels(passes, empty, block, lambda_batch, n_lambda=np.asarray(dv).size)
    if not stats:
        return lev
    return lev, (st[0] if n_test_dirs == 0 else st)


def formal_solve(P_levels, level_map, block, lambda_batch, dv, c_kms, dirs, weights, probes, band=None,
                 method="hum1wei24", i_bc=0.0, want_intensity=False, profile=None):
    """Accelerated CaV result (or the plain one with a single level and all-zero map).

    P_levels: parameter chain (list of [8][nz>>m][nx>>m]); level_map [n_batch][nbz][nbx].
    Each direction is solved separately: eta, chi are evaluated per level from the
    parameters for that direction and handed to the banded (or expanded) plain solver.
    """
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 2)
    weights = np.asarray(weights, dtype=np.float64)
    L = np.asarray(dv).size
    n_probe = np.asarray(probes).size
    J = np.zeros((L, n_probe))
    I = np.zeros((L, dirs.shape[0], n_probe)) if want_intensity else None
    for k in range(dirs.shape[0]):
        wx, wz = -dirs[k, 0], -dirs[k, 1]
        levels = [eta_chi(P, dv, wx, wz, c_kms, method=method, profile=profile) for P in P_levels]
        if band is None:
            e2, c2 = omips.expand(levels, level_map, lambda_batch)
            _, Ik = lc.formal_solve(e2, c2, dirs[k:k + 1], [1.0], probes=probes, i_bc=i_bc, want_intensity=True)
        else:
            _, Ik = lc.formal_solve_banded(levels, level_map, block, lambda_batch, band, dirs[k:k + 1], [1.0],
                                           probes, i_bc=i_bc, want_intensity=True)
        J += weights[k] * Ik[:, 0, :]
        if I is not None:
            I[:, k, :] = Ik[:, 0, :]
    return (J, I) if want_intensity else J
