"""Python binding of the dexgb C ABI: argument marshalling only.

PyTorch provides device memory and streams; every step of the formal solution
runs in the library's CUDA kernels.  Functions mirror the C entry points of
``include/dexgb.h`` (same names without the ``dex_`` prefix).
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._native import DexError, lib

DEX_MAX_DIRS = 256


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Context:
    """A device, a stream and the library's device status word (``dex_ctx``)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = lib().dex_ctx_create(self.device, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise DexError(rc, "dex_ctx_create failed (no usable CUDA device?)")
        self.handle = h

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._rc(lib().dex_ctx_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    def _rc(self, rc: int):
        if rc != 0:
            msg = lib().dex_last_error(self.handle)
            raise DexError(rc, msg.decode() if msg else "")

    def check(self):
        """Synchronise the stream and raise if a kernel recorded an error."""
        self._rc(lib().dex_ctx_check(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().dex_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def planes_floats(n_cells: int, n_lambda: int, W: int) -> int:
    return int(lib().dex_planes_floats(n_cells, n_lambda, W))


def pack_planes(ctx: Context, eta: torch.Tensor, chi: torch.Tensor, W: int, out: torch.Tensor | None = None):
    """eta, chi: float32 CUDA ``[n_lambda][n_cells]`` (any trailing cell shape) ->
    planes ``[n_batch][n_cells][2W]``."""
    n_lambda = eta.shape[0]
    n_cells = eta[0].numel() if n_lambda else 0
    n_batch = -(-n_lambda // W)
    if out is None:
        out = torch.empty((n_batch, n_cells, 2 * W), dtype=torch.float32, device=eta.device)
    ctx._rc(lib().dex_pack_planes(ctx.handle, n_cells, n_lambda, W, _ptr(eta), _ptr(chi), _ptr(out)))
    return out


def _quadrature(dirs, weights):
    d = _host_f32(dirs, (-1, 2))
    w = _host_f32(weights)
    if d.shape[0] != w.size:
        raise ValueError("dirs and weights differ in length")
    return d, w


def formal_solve_dense(ctx: Context, nx: int, nz: int, n_lambda: int, W: int, planes: torch.Tensor,
                       dirs, weights, probes: torch.Tensor | None = None, i_bc: float = 0.0,
                       want_intensity: bool = False, count_segments: bool = False,
                       J: torch.Tensor | None = None):
    """Plain full-resolution long-characteristics solve (``dex_formal_solve_dense``).

    Returns ``(J, I, seg)``: ``J[n_lambda][n_probe]``; ``I[n_lambda][n_dir][n_probe]`` or None;
    a 1-element uint64-as-int64 tensor with the voxel-segment count, or None.
    """
    d, w = _quadrature(dirs, weights)
    dev = planes.device
    n_probe = nx * nz if probes is None else int(probes.numel())
    if J is None:
        J = torch.empty((n_lambda, n_probe), dtype=torch.float32, device=dev)
    I = torch.empty((n_lambda, d.shape[0], n_probe), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_formal_solve_dense(
        ctx.handle, nx, nz, n_lambda, W, _ptr(planes), d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp),
        n_probe, _ptr(probes), float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg
