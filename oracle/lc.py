"""ctypes front end of the float64 long-characteristics oracle (``lc_dense.c``;
the 3D form in ``lc3_dense.c`` is wrapped by ``lc3.py``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the product path.

The C files are compiled with the host ``gcc`` into ``oracle/liboracle.so`` on
first use (or by :func:`build`).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "lc_dense.c"), os.path.join(_HERE, "lc3_dense.c"), os.path.join(_HERE, "rc_dense.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle's C core (gcc, OpenMP) if missing or stale; return the .so path."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_ray_segments.restype = ctypes.c_int
            L.oracle_ray_segments.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int, ip, dp]
            L.oracle_count_segments.restype = ctypes.c_int64
            L.oracle_count_segments.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip]
            L.oracle_formal_solve.restype = ctypes.c_int
            L.oracle_formal_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                              dp, dp, ctypes.c_int, ip, ctypes.c_double, dp, dp]
            L.oracle_formal_solve_banded.restype = ctypes.c_int
            L.oracle_formal_solve_banded.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ip,
                                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                                                     ctypes.c_int, ip, ctypes.c_double, dp, dp]
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_num_threads.argtypes = []
            ci, cd = ctypes.c_int, ctypes.c_double
            L.oracle3_ray_segments.restype = ci
            L.oracle3_ray_segments.argtypes = [ci, ci, ci, cd, cd, cd, cd, cd, cd, ci, ip, dp]
            L.oracle3_count_segments.restype = ctypes.c_int64
            L.oracle3_count_segments.argtypes = [ci, ci, ci, ci, dp, ci, ip]
            L.oracle3_formal_solve.restype = ci
            L.oracle3_formal_solve.argtypes = [ci, ci, ci, ci, dp, dp, ci, dp, dp, ci, ip, cd, dp, dp]
            L.oracle_rc_intervals.restype = ci
            L.oracle_rc_intervals.argtypes = [ci, ci, ci, dp, dp, ci, ci, dp, cd, cd, dp, dp,
                                              ctypes.POINTER(ctypes.c_ubyte)]
            L.oracle3_formal_solve_banded.restype = ci
            L.oracle3_formal_solve_banded.argtypes = [ci, ci, ci, ci, ci, dp, dp, ip, ci, ci, ci, dp, ci, dp, dp,
                                                      ci, ip, cd, dp, dp]
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def ray_segments(nx: int, nz: int, origin, direction):
    """Voxel pieces of one ray from ``origin`` toward ``direction``: (cells j*nx+i, lengths)."""
    cap = 2 * (nx + nz) + 8
    cell = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.float64)
    n = lib().oracle_ray_segments(nx, nz, float(origin[0]), float(origin[1]),
                                  float(direction[0]), float(direction[1]), cap, _iptr(cell), _dptr(ln))
    if n < 0:
        raise RuntimeError("segment capacity exceeded")
    return cell[:n].copy(), ln[:n].copy()


def count_segments(nx: int, nz: int, dirs, probes) -> int:
    """Dense voxel-segment count of all (probe, direction) rays."""
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    return int(lib().oracle_count_segments(nx, nz, d.shape[0], _dptr(d), p.size, _iptr(p)))


def formal_solve(eta, chi, dirs, weights, probes=None, i_bc: float = 0.0, want_intensity: bool = False):
    """Plain float64 formal solution.

    eta, chi: ``[n_lambda][nz][nx]`` (or ``[nz][nx]``).  Returns ``J[n_lambda][n_probe]``
    and, if requested, ``I[n_lambda][n_dir][n_probe]``.  ``probes=None`` means every cell.
    """
    eta = np.asarray(eta, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    if eta.ndim == 2:
        eta, chi = eta[None], chi[None]
    n_lambda, nz, nx = eta.shape
    eta = np.ascontiguousarray(eta)
    chi = np.ascontiguousarray(chi)
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if probes is None:
        probes = np.arange(nx * nz, dtype=np.int32)
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    J = np.zeros((n_lambda, p.size), dtype=np.float64)
    I = np.zeros((n_lambda, d.shape[0], p.size), dtype=np.float64) if want_intensity else None
    rc = lib().oracle_formal_solve(nx, nz, n_lambda, _dptr(eta), _dptr(chi), d.shape[0], _dptr(d), _dptr(w),
                                   p.size, _iptr(p), float(i_bc), _dptr(J),
                                   _dptr(I) if I is not None else ctypes.POINTER(ctypes.c_double)())
    if rc != 0:
        raise RuntimeError("oracle formal solve failed")
    return (J, I) if want_intensity else J


def formal_solve_banded(levels, level_map, block: int, lambda_batch: int, band, dirs, weights, probes,
                        i_bc: float = 0.0, want_intensity: bool = False):
    """Formal solution over MIP levels with a distance-limited level per block visit.

    levels: list of (eta_m, chi_m) ``[L][nz >> m][nx >> m]`` (as from ``mips.mip_chain``);
    level_map: ``[n_batch][nbz][nbx]``; band: thresholds d_1 <= d_2 <= ... (level m allowed
    in blocks entered at t >= d_m).  Returns J (and I) like :func:`formal_solve`.
    """
    L, nz, nx = levels[0][0].shape
    n_lev = len(levels)
    le = np.empty((n_lev, L, nz, nx))
    lch = np.empty((n_lev, L, nz, nx))
    for m, (em, cm) in enumerate(levels):
        f = 2 ** m
        le[m] = np.repeat(np.repeat(em, f, axis=1), f, axis=2)
        lch[m] = np.repeat(np.repeat(cm, f, axis=1), f, axis=2)
    lm = np.ascontiguousarray(np.asarray(level_map, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(band, dtype=np.float64).reshape(-1))
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(probes, dtype=np.int32))
    J = np.zeros((L, p.size))
    I = np.zeros((L, d.shape[0], p.size)) if want_intensity else None
    rc = lib().oracle_formal_solve_banded(nx, nz, L, n_lev, _dptr(le), _dptr(lch), _iptr(lm), block, lambda_batch,
                                          b.size, _dptr(b) if b.size else ctypes.POINTER(ctypes.c_double)(),
                                          d.shape[0], _dptr(d), _dptr(w), p.size, _iptr(p), float(i_bc), _dptr(J),
                                          _dptr(I) if I is not None else ctypes.POINTER(ctypes.c_double)())
    if rc != 0:
        raise RuntimeError("oracle banded formal solve failed")
    return (J, I) if want_intensity else J
