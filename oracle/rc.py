"""Float64 oracle of the radiance-cascade formal solution (2D).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

The paper's code solves the formal solution with radiance cascades around its
traversal (Section 4.1 "Model Configuration"): branching factor 2, so that with
each cascade the probe spacing doubles, the number of directions grows 4x and
the end of the radiance interval moves 4x further from the probe; cascade 0 has
a probe at every voxel, n0 in-plane directions and an interval of 1.5 voxels.
Readings taken here (listed in the design notes):

* cascade i: probe spacing 2^i (probe (px, pz) at (2^i (px + 1/2), 2^i (pz + 1/2))),
  n0 4^i directions theta_k = 2 pi (k + 1/2) / (n0 4^i), interval
  [t0 4^(i-1), t0 4^i] (cascade 0: [0, t0]), t0 = 1.5;
* merge ("vanilla", at the probe position): the radiance of direction k of
  cascade i is L = I + T R, where I, T are the interval's emission and
  transmission and R is, if the ray left the grid inside the interval, the
  boundary intensity; otherwise the bilinear interpolation, at the cascade-i
  probe position, of the mean over directions 4k .. 4k+3 of the merged radiance
  of cascade i + 1 (the 4 nearest cascade-(i+1) probes, indices clamped to the
  lattice at its edges).  The top cascade takes R = i_bc;
* J at cascade-0 probes (every voxel) = the mean over its n0 directions.

The per-interval emission and transmission come from the C core
(``rc_dense.c``); the merge is written out here in numpy.
"""

from __future__ import annotations

import ctypes

import numpy as np

from .lc import _dptr, lib


def geometry(n_cascades: int, n0: int, t0: float = 1.5):
    """Per cascade: (spacing, n_dir, t_s, t_e)."""
    out = []
    for i in range(n_cascades):
        t_s = 0.0 if i == 0 else t0 * 4.0 ** (i - 1)
        out.append((2 ** i, n0 * 4 ** i, t_s, t0 * 4.0 ** i))
    return out


def intervals(eta, chi, spacing: int, dirs, t_s: float, t_e: float):
    """Emission I, transmission T ``[n_dir][pnz][pnx][L]`` and the left-the-grid flag
    ``[n_dir][pnz][pnx]`` of one cascade's radiance intervals."""
    eta = np.ascontiguousarray(np.asarray(eta, dtype=np.float64))
    chi = np.ascontiguousarray(np.asarray(chi, dtype=np.float64))
    L, nz, nx = eta.shape
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
    pnx, pnz = nx // spacing, nz // spacing
    I = np.zeros((d.shape[0], pnz, pnx, L))
    T = np.zeros((d.shape[0], pnz, pnx, L))
    term = np.zeros((d.shape[0], pnz, pnx), dtype=np.uint8)
    rc = lib().oracle_rc_intervals(nx, nz, L, _dptr(eta), _dptr(chi), spacing, d.shape[0], _dptr(d),
                                   float(t_s), float(t_e), _dptr(I), _dptr(T),
                                   term.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    if rc != 0:
        raise RuntimeError("oracle radiance intervals failed")
    return I, T, term.astype(bool)


def _axis_stencil(n_lo: int, n_hi: int):
    """Bilinear stencil along one axis: a probe p of the finer lattice sits at
    u = (p + 1/2)/2 - 1/2 in units of the coarser lattice; returns the two clamped
    coarse indices and the weight of the second."""
    u = (np.arange(n_lo) + 0.5) / 2.0 - 0.5
    q0 = np.floor(u)
    f = u - q0
    i0 = np.clip(q0, 0, n_hi - 1).astype(np.int64)
    i1 = np.clip(q0 + 1, 0, n_hi - 1).astype(np.int64)
    return i0, i1, f


def upper_radiance(upper, n_dir: int, pnz: int, pnx: int):
    """R before the boundary test: bilinear interpolation at the finer probes of the
    mean over each direction's 4 children.  upper ``[4 n_dir][qz][qx][L]``."""
    _, qz, qx, L = upper.shape
    child = upper.reshape(n_dir, 4, qz, qx, L).mean(axis=1)
    z0, z1, fz = _axis_stencil(pnz, qz)
    x0, x1, fx = _axis_stencil(pnx, qx)
    fz = fz[None, :, None, None]
    fx = fx[None, None, :, None]
    c00 = child[:, z0][:, :, x0]
    c01 = child[:, z0][:, :, x1]
    c10 = child[:, z1][:, :, x0]
    c11 = child[:, z1][:, :, x1]
    return (1 - fz) * ((1 - fx) * c00 + fx * c01) + fz * ((1 - fx) * c10 + fx * c11)


def merge(I, T, term, upper, i_bc: float):
    """Merged radiance of one cascade: L = I + T R (R = i_bc where the ray left the grid)."""
    n_dir, pnz, pnx, _ = I.shape
    R = np.full(I.shape, float(i_bc)) if upper is None else upper_radiance(upper, n_dir, pnz, pnx)
    R = np.where(term[..., None], float(i_bc), R)
    return I + T * R


def rc_solve(grids, n_cascades: int, n0: int, dirs, t0: float = 1.5, i_bc: float = 0.0, return_cascades=False):
    """Radiance-cascade J ``[L][nz * nx]`` (cascade-0 probes = every voxel).

    grids: ``(eta, chi)`` ``[L][nz][nx]`` used by every cascade, or a list of one
    ``(eta, chi)`` per cascade (e.g. each cascade's own MIP levels expanded onto
    MIP 0).  dirs: per-cascade direction arrays (``synth.rc_directions``).
    """
    per = grids if isinstance(grids, list) else [grids] * n_cascades
    geo = geometry(n_cascades, n0, t0)
    Lm = None
    merged = []
    for i in reversed(range(n_cascades)):
        spacing, n_dir, t_s, t_e = geo[i]
        I, T, term = intervals(per[i][0], per[i][1], spacing, dirs[i], t_s, t_e)
        Lm = merge(I, T, term, None if i == n_cascades - 1 else Lm, i_bc)
        merged.append(Lm)
    J = Lm.mean(axis=0)                       # [nz][nx][L]
    J = np.moveaxis(J, -1, 0).reshape(J.shape[-1], -1)
    return (J, merged[::-1]) if return_cascades else J
