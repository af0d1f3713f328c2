"""ctypes loader for libdexgb.so (the C ABI declared in include/dexgb.h).

The library is built in-tree by :mod:`paper_2511_08498_gb300.build`.  There is no
fallback: if the library cannot be built or loaded, :func:`lib` raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_float, c_size_t, c_void_p, c_char_p = ctypes.c_int, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p
c_u64p = ctypes.POINTER(ctypes.c_ulonglong)
c_fp = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes); device pointers are passed as c_void_p
PROTOTYPES = {
    "dex_version": (c_int, []),
    "dex_status_string": (c_char_p, [c_int]),
    "dex_ctx_create": (c_int, [c_int, c_void_p, ctypes.POINTER(c_void_p)]),
    "dex_ctx_destroy": (c_int, [c_void_p]),
    "dex_ctx_set_stream": (c_int, [c_void_p, c_void_p]),
    "dex_ctx_set_traversal": (c_int, [c_void_p, c_int]),
    "dex_ctx_set_pair_group": (c_int, [c_void_p, c_int]),
    "dex_ctx_set_own_cell": (c_int, [c_void_p, c_int]),
    "dex_ctx_check": (c_int, [c_void_p]),
    "dex_last_error": (c_char_p, [c_void_p]),
    "dex_planes_floats": (c_size_t, [c_int, c_int, c_int]),
    "dex_pack_planes": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_dense": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_fp, c_fp,
                                       c_int, c_void_p, c_float, c_void_p, c_void_p, c_void_p]),
    "dex_synth_static_line": (c_int, [c_void_p, c_int, c_int] + [c_void_p] * 8),
    "dex_grid_build": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_state_words": (c_size_t, [c_int, c_int]),
    "dex_chain_voxels": (c_int, [c_int]),
    "dex_brick_floats": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "dex_mips_build": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                               c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_hdda": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_int, c_int, c_fp, c_fp, c_int, c_fp, c_float, c_void_p,
                                      c_void_p, c_void_p]),
    "dex_lte_populations": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "dex_atom_eta_chi": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p] + [c_void_p] * 5),
    "dex_rates_accumulate": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
    "dex_se_solve": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 5),
    "dex_mali_rates": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p] + [c_void_p] * 4 +
                       [c_int, c_fp, c_fp, c_void_p, c_void_p]),
    "dex_se_solve_preconditioned": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 6),
    "dex_max_rel_change": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_voigt": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "dex_cav_grid_build": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_cav_brick_floats": (c_size_t, [c_int, c_int]),
    "dex_cav_mips_build": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_fp, c_float, c_void_p, c_void_p,
                                   c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_cav": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_fp, c_float, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_int, c_int, c_fp, c_fp, c_int, c_fp, c_float,
                                     c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_cav_mlp": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_fp, c_float, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_fp, c_fp, c_int,
                                         c_fp, c_float, c_fp, c_void_p, c_void_p, c_void_p]),
    "dex_vel_brick_floats": (c_size_t, [c_int, c_int, c_int, c_int]),
    "dex_vel_mips_build": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int, c_fp, c_float, c_void_p, c_void_p,
                                   c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_velinterp": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                           c_void_p, c_void_p, c_int, c_int, c_fp, c_fp, c_int, c_fp, c_float,
                                           c_void_p, c_void_p, c_void_p]),
    "dex_batch_solve": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "dex_batch_solve_config": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_batch_solve_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "dex_measure_ex2_rate": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "dex_measure_fp32_rate": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "dex_selftest_wait_timeout": (c_int, [c_void_p, c_int]),
    "dex_mlp_param_count": (c_int, []),
    "dex_mlp_forward": (c_int, [c_void_p, ctypes.c_longlong, c_void_p, c_void_p, c_void_p]),
    "dex_mlp_grad": (c_int, [c_void_p, ctypes.c_longlong, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_mlp_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "dex_mlp_targets": (c_int, [c_void_p, ctypes.c_longlong, c_void_p, c_void_p]),
    "dex_rc_workspace_floats": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "dex_rc_solve": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_int,
                             c_int, c_int, c_float, ctypes.POINTER(c_int), c_void_p, c_float, c_void_p, c_void_p,
                             c_void_p]),
    "dex_formal_solve_dense3": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_int, c_fp, c_fp,
                                        c_int, c_void_p, c_float, c_void_p, c_void_p, c_void_p]),
    "dex_grid3_build": (c_int, [c_void_p, c_int, c_int, c_int, c_int] + [c_void_p] * 5),
    "dex_state_words3": (c_size_t, [c_int, c_int, c_int]),
    "dex_chain_voxels3": (c_int, [c_int]),
    "dex_brick3_floats": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "dex_mips3_build": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dex_formal_solve_hdda3": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_int, c_int, c_fp, c_fp, c_int, c_fp, c_float,
                                       c_void_p, c_void_p, c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) libdexgb.so and declare its prototypes."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdexgb.so missing at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class DexError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dexgb error {code}: {msg}")
        self.code = code
