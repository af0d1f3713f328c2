"""ctypes front end of the float64 3D long-characteristics oracle (``lc3_dense.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the product path.

Section 2.3: the traversal and the adapted grid generalise directly to 3D
(cubic blocks, 2x2x2 MIP groups).  Grids are ``[n_lambda][nz][ny][nx]`` with x
fastest; cell index c = (k * ny + j) * nx + i; directions are ``[n_dir][3]``
(d_x, d_y, d_z) unit vectors.
"""

from __future__ import annotations

import ctypes

import numpy as np

from .lc import _dptr, _iptr, lib

_NULL_D = ctypes.POINTER(ctypes.c_double)


def ray_segments(shape, origin, direction):
    """Voxel pieces of one ray in a grid of ``shape = (nx, ny, nz)``: (cells, lengths)."""
    nx, ny, nz = shape
    cap = 3 * (nx + ny + nz) + 8
    cell = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    n = lib().oracle3_ray_segments(nx, ny, nz, *(float(v) for v in origin), *(float(v) for v in direction), cap,
                                   _iptr(cell), _dptr(ln))
    if n < 0:
        raise RuntimeError("segment capacity exceeded")
    return cell[:n].copy(), ln[:n].copy()


def count_segments(shape, dirs, probes) -> int:
    """Full-resolution voxel-segment count of all (probe, direction) rays."""
    nx, ny, nz = shape
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    return int(lib().oracle3_count_segments(nx, ny, nz, d.shape[0], _dptr(d), p.size, _iptr(p)))


def formal_solve(eta, chi, dirs, weights, probes=None, i_bc: float = 0.0, want_intensity: bool = False):
    """Plain float64 formal solution in 3D.

    eta, chi: ``[n_lambda][nz][ny][nx]`` (or ``[nz][ny][nx]``).  Returns
    ``J[n_lambda][n_probe]`` and, if requested, ``I[n_lambda][n_dir][n_probe]``;
    ``probes=None`` means every cell.
    """
    eta = np.asarray(eta, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    if eta.ndim == 3:
        eta, chi = eta[None], chi[None]
    n_lambda, nz, ny, nx = eta.shape
    eta = np.ascontiguousarray(eta)
    chi = np.ascontiguousarray(chi)
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if probes is None:
        probes = np.arange(nx * ny * nz, dtype=np.int32)
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    J = np.zeros((n_lambda, p.size))
    I = np.zeros((n_lambda, d.shape[0], p.size)) if want_intensity else None
    rc = lib().oracle3_formal_solve(nx, ny, nz, n_lambda, _dptr(eta), _dptr(chi), d.shape[0], _dptr(d), _dptr(w),
                                    p.size, _iptr(p), float(i_bc), _dptr(J),
                                    _dptr(I) if I is not None else _NULL_D())
    if rc != 0:
        raise RuntimeError("oracle 3D formal solve failed")
    return (J, I) if want_intensity else J


def upsample(a, f: int):
    """Repeat every voxel of ``[..., Z, Y, X]`` f times along the three grid axes."""
    return np.repeat(np.repeat(np.repeat(a, f, axis=-3), f, axis=-2), f, axis=-1)


def formal_solve_banded(levels, level_map, block: int, lambda_batch: int, band, dirs, weights, probes,
                        i_bc: float = 0.0, want_intensity: bool = False):
    """3D formal solution over MIP levels with a distance-limited level per block visit.

    levels: list of (eta_m, chi_m) ``[L][nz >> m][ny >> m][nx >> m]`` (``mips3.mip_chain``),
    passed at their own resolution; level_map: ``[n_batch][nbz][nby][nbx]``; band:
    thresholds d_1 <= d_2 <= ... (level m allowed in blocks first entered at t >= d_m).
    """
    L, nz, ny, nx = levels[0][0].shape
    n_lev = len(levels)
    le = np.ascontiguousarray(np.concatenate([np.asarray(e, np.float64).reshape(-1) for e, _ in levels]))
    lch = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).reshape(-1) for _, c in levels]))
    lm = np.ascontiguousarray(np.asarray(level_map, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(band, dtype=np.float64).reshape(-1))
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    J = np.zeros((L, p.size))
    I = np.zeros((L, d.shape[0], p.size)) if want_intensity else None
    rc = lib().oracle3_formal_solve_banded(nx, ny, nz, L, n_lev, _dptr(le), _dptr(lch), _iptr(lm), block,
                                           lambda_batch, b.size, _dptr(b) if b.size else _NULL_D(), d.shape[0],
                                           _dptr(d), _dptr(w), p.size, _iptr(p), float(i_bc), _dptr(J),
                                           _dptr(I) if I is not None else _NULL_D())
    if rc != 0:
        raise RuntimeError("oracle 3D banded formal solve failed")
    return (J, I) if want_intensity else J
