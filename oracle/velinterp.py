"""Float64 oracle of the velocity-interpolation treatment of a moving medium (Section 3.1).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

Restated from Section 3.1 with the line model of ``oracle.cav``:
  * every MIP voxel (level m, including MIP 0) carries a uniform grid of n
    projected velocities v_s = -V + 2 V s / (n - 1), s = 0..n-1, where V is the
    largest speed |v| of the MIP-0 cells it contains, and the emissivity and
    opacity at each grid velocity: eta_s = mean over its MIP-0 cells of the cell's
    eta at projected velocity v_s (u = dv + v_s), likewise chi_s;
  * the voxel also keeps its mean velocity (box filter of v_x, v_z);
  * the MIP level of a block per wavelength batch comes from Eq. IoD on the
    rest-frame values (projected velocity 0), with the always-average rule;
  * along a ray (propagation w = -d) a voxel's eta and chi are the linear
    interpolation of its grid at the projected velocity v_mean . w, clamped to
    [-V, V] (the grid is constant when V = 0).
"""

from __future__ import annotations

import numpy as np

from . import lc, mips as omips
from .cav import eta_chi as cav_eta_chi, param_arrays

N_VEL = 8


def _box(a, f):
    """Mean over f x f cells of the trailing two axes."""
    *lead, Z, X = a.shape
    return a.reshape(*lead, Z // f, f, X // f, f).mean(axis=(-3, -1))


def _boxmax(a, f):
    *lead, Z, X = a.shape
    return a.reshape(*lead, Z // f, f, X // f, f).max(axis=(-3, -1))


def velocity_grids(P0, dv, c_kms, max_mip, n_vel=N_VEL, method="hum1wei24"):
    """Per level m: dict(V [nz>>m][nx>>m], vx, vz, eta [n_vel][L][...], chi [n_vel][L][...])."""
    es, cs, a, inv, vx, vz, ec, cc = P0
    speed = np.sqrt(vx * vx + vz * vz)
    out = []
    for m in range(max_mip + 1):
        f = 2 ** m
        V = _boxmax(speed, f)
        Vc = np.repeat(np.repeat(V, f, 0), f, 1)  # each cell sees its voxel's grid
        eta = []
        chi = []
        for s in range(n_vel):
            vs = -Vc + 2.0 * Vc * s / (n_vel - 1)
            # each MIP-0 cell's eta, chi at projected velocity vs (u = dv + vs)
            e, x = _eta_chi_at(P0, dv, vs, c_kms, method)
            eta.append(_box(e, f))
            chi.append(_box(x, f))
        out.append({"V": V, "vx": _box(vx, f), "vz": _box(vz, f), "eta": np.array(eta), "chi": np.array(chi)})
    return out


def _eta_chi_at(P, dv, vproj, c_kms, method):
    """eta, chi [L][...] of cells at a given projected velocity field vproj [...]."""
    es, cs, a, inv, vx, vz, ec, cc = P
    Pz = np.stack([es, cs, a, inv, np.ones_like(vx), np.zeros_like(vz), ec, cc])
    # v . w = vproj with w = (1, 0) and v_x = vproj
    Pz[4] = vproj
    return cav_eta_chi(Pz, dv, 1.0, 0.0, c_kms, method=method)


def rest_frame(P0, dv, c_kms, method="hum1wei24"):
    return cav_eta_chi(P0, dv, 0.0, 0.0, c_kms, method=method)


def interpolate(grid, wx, wz):
    """eta, chi [L][...] of every voxel of one level for propagation (wx, wz)."""
    V = grid["V"]
    n_vel = grid["eta"].shape[0]
    proj = grid["vx"] * wx + grid["vz"] * wz
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(V > 0, (np.clip(proj, -V, V) + V) / (2.0 * np.where(V > 0, V, 1.0)) * (n_vel - 1), 0.0)
    i0 = np.minimum(np.floor(f).astype(int), n_vel - 2)
    t = f - i0
    take = lambda arr, idx: np.take_along_axis(arr, np.broadcast_to(idx[None, None], (1,) + arr.shape[1:]), 0)[0]
    e = (1 - t) * take(grid["eta"], i0) + t * take(grid["eta"], i0 + 1)
    x = (1 - t) * take(grid["chi"], i0) + t * take(grid["chi"], i0 + 1)
    return e, x


def formal_solve(grids, level_map, block, lambda_batch, dirs, weights, probes, band=None, want_intensity=False):
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 2)
    weights = np.asarray(weights, dtype=np.float64)
    L = grids[0]["eta"].shape[1]
    n_probe = np.asarray(probes).size
    J = np.zeros((L, n_probe))
    I = np.zeros((L, dirs.shape[0], n_probe)) if want_intensity else None
    for k in range(dirs.shape[0]):
        levels = [interpolate(g, -dirs[k, 0], -dirs[k, 1]) for g in grids]
        if band is None:
            e2, c2 = omips.expand(levels, level_map, lambda_batch)
            _, Ik = lc.formal_solve(e2, c2, dirs[k:k + 1], [1.0], probes=probes, want_intensity=True)
        else:
            _, Ik = lc.formal_solve_banded(levels, level_map, block, lambda_batch, band, dirs[k:k + 1], [1.0],
                                           probes, want_intensity=True)
        J += weights[k] * Ik[:, 0, :]
        if I is not None:
            I[:, k, :] = Ik[:, 0, :]
    return (J, I) if want_intensity else J


def levels(P0, dv, c_kms, empty, block, lambda_batch, max_mip, thr, chi_ds_min=0.25, stats=False, n_test_dirs=0):
    """Per-batch block levels from the rest-frame IoD test (Section 3.1).

    With ``n_test_dirs`` = K > 0 a group must also pass the same test on its
    children's velocity grids interpolated as a ray propagating along each
    w_k = (cos 2 pi k / K, sin 2 pi k / K) samples them (a reading, as in
    ``oracle.cav.block_levels``); ``stats`` as there."""
    e0, x0 = rest_frame(P0, dv, c_kms)
    res = omips.mip_chain(e0, x0, max_mip, thr, thr, chi_ds_min, mean="linear", stats=True)
    passes = list(res[1])
    st_all = [res[2]]
    if n_test_dirs > 0 and max_mip > 0:
        from .cav import test_directions
        grids = velocity_grids(P0, dv, c_kms, max_mip - 1)
        for wx, wz in test_directions(n_test_dirs):
            st_d = []
            for m in range(1, max_mip + 1):
                ds = float(2 ** m)
                e, x = interpolate(grids[m - 1], wx, wz)
                ge, gx = omips._groups(e), omips._groups(x)
                _, iod_e = omips._reduce(ge, ds, "linear")
                _, iod_c = omips._reduce(gx, ds, "linear")
                kds = gx.max(-1) * ds
                passes[m - 1] = passes[m - 1] & (((iod_e < thr) & (iod_c < thr)) | (kds < chi_ds_min))
                st_d.append({"iod_eta": iod_e, "iod_chi": iod_c, "chi_ds": kds})
            st_all.append(st_d)
    lev = omips.block_levels(passes, empty, block, lambda_batch, n_lambda=np.asarray(dv).size)
    if not stats:
        return lev
    return lev, (st_all[0] if n_test_dirs == 0 else st_all)
