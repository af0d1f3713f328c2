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
# traversal modes of the static accelerated solve (dex_ctx_set_traversal)
TRAVERSAL_PER_BATCH, TRAVERSAL_SHARED, TRAVERSAL_PAIRED = 0, 1, 2


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

    def set_traversal(self, mode):
        """Static accelerated solve at W = 8 (``dex_ctx_set_traversal``): one walk per
        ray and wavelength batch (``TRAVERSAL_PER_BATCH`` or False, the default), one
        walk for two batches at their own levels (``TRAVERSAL_SHARED`` or True), or one
        walk for the pair of batches b, n_batch - 1 - b on the smaller of their levels,
        one thread carrying 16 wavelengths (``TRAVERSAL_PAIRED``)."""
        if isinstance(mode, bool):
            mode = TRAVERSAL_SHARED if mode else TRAVERSAL_PER_BATCH
        self._rc(lib().dex_ctx_set_traversal(self.handle, int(mode)))

    def set_pair_group(self, group: int):
        """Pairs of the paired walk: mirror-wise within consecutive groups of
        ``group`` wavelength batches, 0 for one group of all (``dex_ctx_set_pair_group``)."""
        self._rc(lib().dex_ctx_set_pair_group(self.handle, int(group)))

    def set_own_cell(self, include: bool):
        """Include (default) or leave out each probe's own-cell emission in the
        plain and accelerated solves (``dex_ctx_set_own_cell``)."""
        self._rc(lib().dex_ctx_set_own_cell(self.handle, 1 if include else 0))

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
    n_probe_arg = -1 if probes is None else n_probe
    if J is None:
        J = torch.empty((n_lambda, n_probe), dtype=torch.float32, device=dev)
    I = torch.empty((n_lambda, d.shape[0], n_probe), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_formal_solve_dense(
        ctx.handle, nx, nz, n_lambda, W, _ptr(planes), d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp),
        n_probe_arg, _ptr(probes) if n_probe_arg > 0 else None, float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


# ------------------------------------------------------------ sparse path --

BLOCK = 16
STATES_PER_WORD = 21


class VlmParams(ctypes.Structure):
    """``dex_vlm_params``: variance-limited mipmapping thresholds (Section 2.2)."""
    _fields_ = [("iod_eta", ctypes.c_float), ("iod_chi", ctypes.c_float), ("chi_ds_min", ctypes.c_float),
                ("max_mip", ctypes.c_int), ("log_mean", ctypes.c_int), ("storage", ctypes.c_int),
                ("n_test_dirs", ctypes.c_int)]


STORE_F32, STORE_BF16, STORE_F16 = 0, 1, 2


class SparseGrid:
    """Block sparsity map and Morton layout (device tensors) of an nx x nz grid."""

    def __init__(self, nx, nz, block_offset, active, n_active):
        self.nx, self.nz = nx, nz
        self.nbx, self.nbz = nx // BLOCK, nz // BLOCK
        self.block_offset = block_offset
        self.active = active
        self.n_active_dev = n_active

    @property
    def n_blocks(self):
        return self.nbx * self.nbz

    def n_active(self) -> int:
        """Number of active blocks (synchronises)."""
        return int(self.n_active_dev.item())


class Mips:
    """MIP chain bricks and packed block states of every wavelength batch."""

    def __init__(self, bricks, words, W, max_mip, n_lambda, capacity, storage=0):
        self.bricks, self.words = bricks, words
        self.W, self.max_mip, self.n_lambda, self.capacity = W, max_mip, n_lambda, capacity
        self.storage = storage


def synth_static_line(ctx: Context, chi_c, s_c, s_l, ratio, dld, dlam, eta=None, chi=None):
    """MIP-0 eta, chi ``[n_lambda][n_cells]`` of the continuum + line model (``dex_synth_static_line``)."""
    n_cells = chi_c.numel()
    n_lambda = dlam.numel()
    if eta is None:
        eta = torch.empty((n_lambda, n_cells), dtype=torch.float32, device=chi_c.device)
    if chi is None:
        chi = torch.empty((n_lambda, n_cells), dtype=torch.float32, device=chi_c.device)
    ctx._rc(lib().dex_synth_static_line(ctx.handle, n_cells, n_lambda, _ptr(chi_c), _ptr(s_c), _ptr(s_l),
                                        _ptr(ratio), _ptr(dld), _ptr(dlam), _ptr(eta), _ptr(chi)))
    return eta, chi


def grid_build(ctx: Context, nx: int, nz: int, eta: torch.Tensor, chi: torch.Tensor, out: SparseGrid | None = None):
    """Sparsity map + Morton-ordered active blocks (``dex_grid_build``); no synchronisation."""
    n_lambda = eta.shape[0]
    nb = (nx // BLOCK) * (nz // BLOCK)
    if out is None:
        dev = eta.device
        out = SparseGrid(nx, nz, torch.empty(nb, dtype=torch.int32, device=dev),
                         torch.zeros(nb, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int32, device=dev))
    ctx._rc(lib().dex_grid_build(ctx.handle, nx, nz, n_lambda, _ptr(eta), _ptr(chi), _ptr(out.block_offset),
                                 _ptr(out.active), _ptr(out.n_active_dev)))
    return out


def state_words(nx: int, nz: int) -> int:
    return int(lib().dex_state_words(nx, nz))


def chain_voxels(max_mip: int) -> int:
    return int(lib().dex_chain_voxels(max_mip))


def mips_build(ctx: Context, grid: SparseGrid, eta, chi, W: int, max_mip: int, iod_eta: float, iod_chi: float,
               chi_ds_min: float = 0.25, log_mean: bool = False, level_cap: torch.Tensor | None = None,
               capacity: int | None = None, out: Mips | None = None, storage: int = STORE_F32):
    """MIP chains + VLM block levels of every wavelength batch (``dex_mips_build``).

    ``storage``: record format of the bricks (STORE_F32, STORE_BF16, STORE_F16)."""
    n_lambda = eta.shape[0]
    cap = grid.n_blocks if capacity is None else int(capacity)
    n_batch = -(-n_lambda // W)
    if out is None:
        nf = int(lib().dex_brick_floats(cap, n_lambda, W, max_mip, storage))
        bricks = torch.empty(max(nf, 4), dtype=torch.float32, device=eta.device)
        words = torch.empty((n_batch, state_words(grid.nx, grid.nz)), dtype=torch.int64, device=eta.device)
        out = Mips(bricks, words, W, max_mip, n_lambda, cap, storage)
    p = VlmParams(float(iod_eta), float(iod_chi), float(chi_ds_min), int(max_mip), 1 if log_mean else 0,
                  int(out.storage))
    ctx._rc(lib().dex_mips_build(ctx.handle, grid.nx, grid.nz, n_lambda, W, _ptr(eta), _ptr(chi), _ptr(grid.active),
                                 _ptr(grid.n_active_dev), cap, ctypes.byref(p), _ptr(level_cap), _ptr(out.bricks),
                                 _ptr(out.words)))
    return out


def formal_solve_hdda(ctx: Context, grid: SparseGrid, mips: Mips, dirs, weights, i_bc: float = 0.0,
                      want_intensity: bool = False, count_segments: bool = False, J: torch.Tensor | None = None,
                      band=None):
    """Accelerated (sparse + mipmapped) solve (``dex_formal_solve_hdda``).

    ``band``: optional non-decreasing distances (at most 4); level m is used only in
    blocks first entered at ray parameter t >= band[m-1].

    Returns ``(J, I, seg)`` with dense ``J[n_lambda][nz*nx]`` (zero outside active blocks),
    optional ``I[n_lambda][n_dir][nz*nx]`` and the integrated-segment count.
    """
    d, w = _quadrature(dirs, weights)
    dev = mips.bricks.device
    n_cells = grid.nx * grid.nz
    if J is None:
        J = torch.empty((mips.n_lambda, n_cells), dtype=torch.float32, device=dev)
    I = torch.empty((mips.n_lambda, d.shape[0], n_cells), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    b = None if band is None else _host_f32(band).reshape(-1)
    ctx._rc(lib().dex_formal_solve_hdda(
        ctx.handle, grid.nx, grid.nz, mips.n_lambda, mips.W, mips.max_mip, int(mips.storage), _ptr(mips.bricks),
        _ptr(mips.words), _ptr(grid.block_offset), _ptr(grid.active), _ptr(grid.n_active_dev), mips.capacity,
        d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp), -1 if b is None else b.size,
        None if b is None else b.ctypes.data_as(fp), float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


def unpack_states(words: np.ndarray, n_blocks: int) -> np.ndarray:
    """Host-side decode of packed block states into levels (-1 = empty), for inspection."""
    w = np.asarray(words).astype(np.uint64).reshape(-1, words.shape[-1])
    out = np.empty((w.shape[0], n_blocks), dtype=np.int32)
    k = np.arange(n_blocks)
    for b in range(w.shape[0]):
        out[b] = ((w[b][k // STATES_PER_WORD] >> (3 * (k % STATES_PER_WORD)).astype(np.uint64)) & 7).astype(np.int32) - 1
    return out


# ---------------------------------------------------- level populations --

MAX_LEVELS, MAX_LINES = 4, 4


class Atom(ctypes.Structure):
    """``dex_atom``: levels, radiative lines and collision strengths (cgs)."""
    _fields_ = [("n_level", ctypes.c_int), ("energy_erg", ctypes.c_double * MAX_LEVELS),
                ("g", ctypes.c_double * MAX_LEVELS), ("n_line", ctypes.c_int),
                ("line_lower", ctypes.c_int * MAX_LINES), ("line_upper", ctypes.c_int * MAX_LINES),
                ("line_A", ctypes.c_double * MAX_LINES), ("line_lambda0_nm", ctypes.c_double * MAX_LINES),
                ("upsilon", (ctypes.c_double * MAX_LEVELS) * MAX_LEVELS), ("mass_amu", ctypes.c_double),
                ("background_sigma", ctypes.c_double), ("cell_cm", ctypes.c_double)]

    @classmethod
    def from_dict(cls, d, cell_cm: float, background_sigma: float = 6.652e-25):
        a = cls()
        ev = 1.602176634e-12
        a.n_level = len(d["g"])
        for i, (E, g) in enumerate(zip(d["energy_ev"], d["g"])):
            a.energy_erg[i] = float(E) * ev
            a.g[i] = float(g)
        a.n_line = len(d["lines"])
        for l, (lo, up, A, lam0) in enumerate(d["lines"]):
            a.line_lower[l], a.line_upper[l], a.line_A[l], a.line_lambda0_nm[l] = lo, up, A, lam0
        for (i, j), u in d["upsilon"].items():
            a.upsilon[i][j] = float(u)
        a.mass_amu = float(d["mass_amu"])
        a.background_sigma = float(background_sigma)
        a.cell_cm = float(cell_cm)
        return a


def _lam_arrays(lam_nm, tag):
    lam = np.ascontiguousarray(np.asarray(lam_nm, dtype=np.float64))
    tg = np.ascontiguousarray(np.asarray(tag, dtype=np.int32))
    return lam, tg, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), tg.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def lte_populations(ctx: Context, atom: Atom, T, nh, out=None):
    n = T.numel()
    if out is None:
        out = torch.empty((atom.n_level, n), dtype=torch.float64, device=T.device)
    ctx._rc(lib().dex_lte_populations(ctx.handle, ctypes.byref(atom), n, _ptr(T), _ptr(nh), _ptr(out)))
    return out


def atom_eta_chi(ctx: Context, atom: Atom, lam_nm, tag, T, ne, pops, eta=None, chi=None):
    n = T.numel()
    lam, tg, lp, tp = _lam_arrays(lam_nm, tag)
    if eta is None:
        eta = torch.empty((lam.size, n), dtype=torch.float32, device=T.device)
    if chi is None:
        chi = torch.empty((lam.size, n), dtype=torch.float32, device=T.device)
    ctx._rc(lib().dex_atom_eta_chi(ctx.handle, ctypes.byref(atom), n, lam.size, lp, tp, _ptr(T), _ptr(ne), _ptr(pops),
                                   _ptr(eta), _ptr(chi)))
    return eta, chi


def rates_accumulate(ctx: Context, atom: Atom, lam_nm, tag, T, J, out=None):
    n = T.numel()
    lam, tg, lp, tp = _lam_arrays(lam_nm, tag)
    if out is None:
        out = torch.empty((max(atom.n_line, 1), n), dtype=torch.float64, device=T.device)
    ctx._rc(lib().dex_rates_accumulate(ctx.handle, ctypes.byref(atom), n, lam.size, lp, tp, _ptr(T), _ptr(J),
                                       _ptr(out)))
    return out


def se_solve(ctx: Context, atom: Atom, T, ne, nh, jbar, out=None):
    n = T.numel()
    if out is None:
        out = torch.empty((atom.n_level, n), dtype=torch.float64, device=T.device)
    ctx._rc(lib().dex_se_solve(ctx.handle, ctypes.byref(atom), n, _ptr(T), _ptr(ne), _ptr(nh), _ptr(jbar),
                               _ptr(out)))
    return out


def lambda_iteration(ctx: Context, atom: Atom, lam_nm, tag, T, ne, nh, nx: int, nz: int, dirs, weights,
                     n_iter: int, accelerated: bool = False, W: int = 8, max_mip: int = 3, iod: float = 1e-2,
                     chi_ds_min: float = 0.25, band=None, pops=None, storage: int = STORE_F32,
                     cascades: dict | None = None):
    """Fixed-length Lambda iteration: [eta, chi -> formal solution -> Jbar -> SE] x n_iter.

    Every step is a library call; this function only sequences them.  The plain
    variant solves at full resolution from every cell of every non-empty block
    (``dex_formal_solve_dense`` over that probe list); the accelerated one builds
    the MIP chains (records in the ``storage`` format) and runs the HDDA solve.
    With ``cascades`` (keys ``n_cascades``, ``n0``, optional ``t0``,
    ``level_cap``) the formal solution is the radiance-cascade solve instead
    (``dirs``/``weights`` unused): at full resolution when not ``accelerated``,
    else over the VLM levels with the per-cascade caps.
    Returns the float64 populations.
    """
    n = nx * nz
    L = int(np.asarray(lam_nm).size)
    if pops is None:
        pops = lte_populations(ctx, atom, T, nh)
    eta = torch.empty((L, n), dtype=torch.float32, device=T.device)
    chi = torch.empty_like(eta)
    J = torch.empty_like(eta)
    jbar = None
    grid, mips, planes, probes = None, None, None, None
    rc_ws = None
    for _ in range(n_iter):
        atom_eta_chi(ctx, atom, lam_nm, tag, T, ne, pops, eta, chi)
        grid = grid_build(ctx, nx, nz, eta, chi, out=grid)
        if cascades is not None:
            C, n0 = int(cascades["n_cascades"]), int(cascades["n0"])
            if rc_ws is None:
                rc_ws = torch.empty(max(rc_workspace_floats(nx, nz, L, W, n0), 4), dtype=torch.float32,
                                    device=T.device)
            mm = max_mip if accelerated else 0
            mips = mips_build(ctx, grid, eta, chi, W, mm, iod, iod, chi_ds_min, out=mips, storage=storage)
            caps = cascades.get("level_cap") if accelerated else [0] * C
            rc_solve(ctx, grid, mips, C, n0, float(cascades.get("t0", 1.5)), level_cap=caps, J=J, workspace=rc_ws)
        elif accelerated:
            mips = mips_build(ctx, grid, eta, chi, W, max_mip, iod, iod, chi_ds_min, out=mips, storage=storage)
            formal_solve_hdda(ctx, grid, mips, dirs, weights, J=J, band=band)
        else:
            if probes is None:
                off = grid.block_offset.view(grid.nbz, grid.nbx) >= 0
                cell = off.repeat_interleave(BLOCK, 0).repeat_interleave(BLOCK, 1).reshape(-1)
                probes = torch.nonzero(cell).to(torch.int32).reshape(-1)
                Jp = torch.empty((L, probes.numel()), dtype=torch.float32, device=T.device)
            planes = pack_planes(ctx, eta, chi, W, out=planes)
            formal_solve_dense(ctx, nx, nz, L, W, planes, dirs, weights, probes=probes, J=Jp)
            J.zero_()
            J[:, probes.long()] = Jp
        jbar = rates_accumulate(ctx, atom, lam_nm, tag, T, J, out=jbar)
        pops = se_solve(ctx, atom, T, ne, nh, jbar, out=pops)
    return pops


def mali_rates(ctx: Context, atom: Atom, lam_nm, tag, T, ne, pops, Jext, dirs, weights, rho=None, jeff=None):
    """``dex_mali_rates``: (rho = 1 - Psibar, Jbar_eff) per line and cell, float64,
    from the populations and the formal solution without the own-cell emission."""
    n = T.numel()
    lam, tg, lp, tp = _lam_arrays(lam_nm, tag)
    d, w = _quadrature(dirs, weights)
    shape = (max(atom.n_line, 1), n)
    rho = torch.empty(shape, dtype=torch.float64, device=T.device) if rho is None else rho
    jeff = torch.empty(shape, dtype=torch.float64, device=T.device) if jeff is None else jeff
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_mali_rates(ctx.handle, ctypes.byref(atom), n, lam.size, lp, tp, _ptr(T), _ptr(ne), _ptr(pops),
                                 _ptr(Jext), d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp), _ptr(rho),
                                 _ptr(jeff)))
    return rho, jeff


def se_solve_preconditioned(ctx: Context, atom: Atom, T, ne, nh, rho, jeff, out=None):
    """``dex_se_solve_preconditioned``: the MALI populations from the preconditioned rates."""
    n = T.numel()
    if out is None:
        out = torch.empty((atom.n_level, n), dtype=torch.float64, device=T.device)
    ctx._rc(lib().dex_se_solve_preconditioned(ctx.handle, ctypes.byref(atom), n, _ptr(T), _ptr(ne), _ptr(nh),
                                              _ptr(rho), _ptr(jeff), _ptr(out)))
    return out


def max_rel_change(ctx: Context, T, old, new, out=None):
    """``dex_max_rel_change`` into a 1-element float64 device tensor."""
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=T.device)
    ctx._rc(lib().dex_max_rel_change(ctx.handle, int(old.shape[0]), T.numel(), _ptr(T), _ptr(old), _ptr(new),
                                     _ptr(out)))
    return out


def mali_iteration(ctx: Context, atom: Atom, lam_nm, tag, T, ne, nh, nx: int, nz: int, dirs, weights,
                   tol: float = 1e-3, max_iter: int = 200, accelerated: bool = False, W: int = 8, max_mip: int = 3,
                   iod: float = 1e-2, chi_ds_min: float = 0.25, band=None, storage: int = STORE_F32,
                   n_iter: int | None = None):
    """MALI from LTE (Section 4.1): [eta, chi -> formal solution -> preconditioned
    rates -> SE] until the largest relative population change is below ``tol``
    (or exactly ``n_iter`` updates when given).

    Every step is a library call; this function only sequences them (the formal
    solution as in :func:`lambda_iteration`) and reads one number per iteration,
    the convergence measure.  Returns ``(pops, n_updates, history)``.
    """
    n = nx * nz
    L = int(np.asarray(lam_nm).size)
    pops = lte_populations(ctx, atom, T, nh)
    new = torch.empty_like(pops)
    eta = torch.empty((L, n), dtype=torch.float32, device=T.device)
    chi = torch.empty_like(eta)
    J = torch.empty_like(eta)
    rho = jeff = None
    grid = mips = planes = probes = Jp = None
    change = torch.empty(1, dtype=torch.float64, device=T.device)
    hist = []
    limit = max_iter if n_iter is None else n_iter
    for it in range(limit):
        atom_eta_chi(ctx, atom, lam_nm, tag, T, ne, pops, eta, chi)
        grid = grid_build(ctx, nx, nz, eta, chi, out=grid)
        ctx.set_own_cell(False)   # the solves return Jext
        try:
            if accelerated:
                mips = mips_build(ctx, grid, eta, chi, W, max_mip, iod, iod, chi_ds_min, out=mips, storage=storage)
                formal_solve_hdda(ctx, grid, mips, dirs, weights, J=J, band=band)
            else:
                if probes is None:
                    off = grid.block_offset.view(grid.nbz, grid.nbx) >= 0
                    cell = off.repeat_interleave(BLOCK, 0).repeat_interleave(BLOCK, 1).reshape(-1)
                    probes = torch.nonzero(cell).to(torch.int32).reshape(-1)
                    Jp = torch.empty((L, probes.numel()), dtype=torch.float32, device=T.device)
                planes = pack_planes(ctx, eta, chi, W, out=planes)
                formal_solve_dense(ctx, nx, nz, L, W, planes, dirs, weights, probes=probes, J=Jp)
                J.zero_()
                J[:, probes.long()] = Jp
        finally:
            ctx.set_own_cell(True)
        rho, jeff = mali_rates(ctx, atom, lam_nm, tag, T, ne, pops, J, dirs, weights, rho=rho, jeff=jeff)
        new = se_solve_preconditioned(ctx, atom, T, ne, nh, rho, jeff, out=new)
        max_rel_change(ctx, T, pops, new, out=change)
        hist.append(float(change.item()))
        pops, new = new, pops
        if n_iter is None and hist[-1] < tol:
            return pops, it + 1, hist
    return pops, limit, hist


def voigt(ctx: Context, a: torch.Tensor, x: torch.Tensor, out=None):
    """H(a, x) by HUM1WEI24 (``dex_voigt``); a, x float32 CUDA tensors of equal size."""
    if out is None:
        out = torch.empty_like(x)
    ctx._rc(lib().dex_voigt(ctx.handle, x.numel(), _ptr(a), _ptr(x), _ptr(out)))
    return out


# --------------------------------------------------------- Core and Voigt --

CAV_FIELDS = ("eta_star", "chi_star", "damping", "vth", "vx", "vz", "eta_c", "chi_c")


class CavFields(ctypes.Structure):
    """``dex_cav_fields``: device pointers of the 8 per-cell CaV fields."""
    _fields_ = [(k, ctypes.c_void_p) for k in CAV_FIELDS]

    @classmethod
    def from_tensors(cls, t: dict):
        return cls(*[t[k].data_ptr() for k in CAV_FIELDS])


class CavMips:
    def __init__(self, bricks, words, W, max_mip, dv, c_kms, capacity):
        self.bricks, self.words, self.W, self.max_mip = bricks, words, W, max_mip
        self.dv = np.ascontiguousarray(np.asarray(dv, dtype=np.float32))
        self.c_kms, self.capacity = float(c_kms), capacity
        self.n_lambda = self.dv.size


def cav_grid_build(ctx: Context, nx: int, nz: int, fields: dict, out: SparseGrid | None = None):
    nb = (nx // BLOCK) * (nz // BLOCK)
    dev = fields["chi_c"].device
    if out is None:
        out = SparseGrid(nx, nz, torch.empty(nb, dtype=torch.int32, device=dev),
                         torch.zeros(nb, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int32, device=dev))
    f = CavFields.from_tensors(fields)
    ctx._rc(lib().dex_cav_grid_build(ctx.handle, nx, nz, ctypes.byref(f), _ptr(out.block_offset), _ptr(out.active),
                                     _ptr(out.n_active_dev)))
    return out


def cav_mips_build(ctx: Context, grid: SparseGrid, fields: dict, dv, c_kms: float, W: int, max_mip: int,
                   iod_eta: float, iod_chi: float, chi_ds_min: float = 0.25, level_cap=None, capacity=None,
                   out: CavMips | None = None, test_dirs: int = 0):
    cap = grid.n_blocks if capacity is None else int(capacity)
    dvh = np.ascontiguousarray(np.asarray(dv, dtype=np.float32))
    n_batch = -(-dvh.size // W)
    dev = fields["chi_c"].device
    if out is None:
        nf = int(lib().dex_cav_brick_floats(cap, max_mip))
        out = CavMips(torch.empty(max(nf, 4), dtype=torch.float32, device=dev),
                      torch.empty((n_batch, state_words(grid.nx, grid.nz)), dtype=torch.int64, device=dev),
                      W, max_mip, dvh, c_kms, cap)
    f = CavFields.from_tensors(fields)
    p = VlmParams(float(iod_eta), float(iod_chi), float(chi_ds_min), int(max_mip), 0, STORE_F32, int(test_dirs))
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_cav_mips_build(ctx.handle, grid.nx, grid.nz, ctypes.byref(f), dvh.size, W,
                                     dvh.ctypes.data_as(fp), float(c_kms), _ptr(grid.active), _ptr(grid.n_active_dev),
                                     cap, ctypes.byref(p), _ptr(level_cap), _ptr(out.bricks), _ptr(out.words)))
    return out


def formal_solve_cav(ctx: Context, grid: SparseGrid, mips: CavMips, dirs, weights, band=None, i_bc: float = 0.0,
                     want_intensity: bool = False, count_segments: bool = False, J: torch.Tensor | None = None,
                     mlp_params=None):
    """Core-and-Voigt solve (``dex_formal_solve_cav``); outputs as :func:`formal_solve_hdda`.

    ``mlp_params`` (the surrogate network's parameters, any array-like; copied to
    the host) selects ``dex_formal_solve_cav_mlp``: the network as the profile
    inside its training domain, the exact evaluation outside it."""
    d, w = _quadrature(dirs, weights)
    dev = mips.bricks.device
    n_cells = grid.nx * grid.nz
    L = mips.n_lambda
    if J is None:
        J = torch.empty((L, n_cells), dtype=torch.float32, device=dev)
    I = torch.empty((L, d.shape[0], n_cells), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    b = None if band is None else _host_f32(band).reshape(-1)
    common = (ctx.handle, grid.nx, grid.nz, L, mips.W, mips.max_mip, mips.dv.ctypes.data_as(fp), mips.c_kms,
              _ptr(mips.bricks), _ptr(mips.words), _ptr(grid.block_offset), _ptr(grid.active),
              _ptr(grid.n_active_dev), mips.capacity, d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp),
              -1 if b is None else b.size, None if b is None else b.ctypes.data_as(fp), float(i_bc))
    if mlp_params is None:
        ctx._rc(lib().dex_formal_solve_cav(*common, _ptr(J), _ptr(I), _ptr(seg)))
    else:
        if isinstance(mlp_params, torch.Tensor):
            mlp_params = mlp_params.detach().cpu().numpy()
        net = _host_f32(mlp_params).reshape(-1)
        if net.size != mlp_param_count():
            raise ValueError(f"expected {mlp_param_count()} network parameters, got {net.size}")
        ctx._rc(lib().dex_formal_solve_cav_mlp(*common, net.ctypes.data_as(fp), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


# ------------------------------------------------- velocity interpolation --

VEL_SAMPLES = 8


def vel_mips_build(ctx: Context, grid: SparseGrid, fields: dict, dv, c_kms: float, W: int, max_mip: int,
                   iod_eta: float, iod_chi: float, chi_ds_min: float = 0.25, level_cap=None, capacity=None,
                   out: CavMips | None = None, test_dirs: int = 0):
    """Velocity-grid MIP chains + rest-frame VLM levels (``dex_vel_mips_build``)."""
    cap = grid.n_blocks if capacity is None else int(capacity)
    dvh = np.ascontiguousarray(np.asarray(dv, dtype=np.float32))
    n_batch = -(-dvh.size // W)
    dev = fields["chi_c"].device
    if out is None:
        nf = int(lib().dex_vel_brick_floats(cap, dvh.size, W, max_mip))
        out = CavMips(torch.empty(max(nf, 4), dtype=torch.float32, device=dev),
                      torch.empty((n_batch, state_words(grid.nx, grid.nz)), dtype=torch.int64, device=dev),
                      W, max_mip, dvh, c_kms, cap)
    f = CavFields.from_tensors(fields)
    p = VlmParams(float(iod_eta), float(iod_chi), float(chi_ds_min), int(max_mip), 0, STORE_F32, int(test_dirs))
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_vel_mips_build(ctx.handle, grid.nx, grid.nz, ctypes.byref(f), dvh.size, W,
                                     dvh.ctypes.data_as(fp), float(c_kms), _ptr(grid.active), _ptr(grid.n_active_dev),
                                     cap, ctypes.byref(p), _ptr(level_cap), _ptr(out.bricks), _ptr(out.words)))
    return out


def formal_solve_velinterp(ctx: Context, grid: SparseGrid, mips: CavMips, dirs, weights, band=None,
                           i_bc: float = 0.0, want_intensity: bool = False, count_segments: bool = False,
                           J: torch.Tensor | None = None):
    """Velocity-interpolation solve (``dex_formal_solve_velinterp``)."""
    d, w = _quadrature(dirs, weights)
    dev = mips.bricks.device
    n_cells = grid.nx * grid.nz
    L = mips.n_lambda
    if J is None:
        J = torch.empty((L, n_cells), dtype=torch.float32, device=dev)
    I = torch.empty((L, d.shape[0], n_cells), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    b = None if band is None else _host_f32(band).reshape(-1)
    ctx._rc(lib().dex_formal_solve_velinterp(
        ctx.handle, grid.nx, grid.nz, L, mips.W, mips.max_mip, _ptr(mips.bricks), _ptr(mips.words),
        _ptr(grid.block_offset), _ptr(grid.active), _ptr(grid.n_active_dev), mips.capacity, d.shape[0],
        d.ctypes.data_as(fp), w.ctypes.data_as(fp), -1 if b is None else b.size,
        None if b is None else b.ctypes.data_as(fp), float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


# ---------------------------------------------------- batched atmospheres --

MAX_BATCH_ATM = 32


class BatchItem(ctypes.Structure):
    """``dex_batch_item``: one atmosphere of a batched solve (device pointers inside)."""
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("n_lambda", ctypes.c_int), ("max_mip", ctypes.c_int),
                ("capacity", ctypes.c_int), ("bricks", ctypes.c_void_p), ("state_words", ctypes.c_void_p),
                ("block_offset", ctypes.c_void_p), ("active", ctypes.c_void_p), ("n_active", ctypes.c_void_p),
                ("n_dir", ctypes.c_int), ("dirs", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n_band", ctypes.c_int), ("band", ctypes.c_float * 4), ("i_bc", ctypes.c_float),
                ("J", ctypes.c_void_p)]


def batch_item(grid: SparseGrid, mips: Mips, dirs_dev: torch.Tensor, weights_dev: torch.Tensor, J: torch.Tensor,
               band=None, i_bc: float = 0.0) -> BatchItem:
    if getattr(mips, "storage", STORE_F32) != STORE_F32:
        raise ValueError("the batched solve reads float32 bricks")
    it = BatchItem()
    it.nx, it.nz, it.n_lambda, it.max_mip, it.capacity = grid.nx, grid.nz, mips.n_lambda, mips.max_mip, mips.capacity
    it.bricks, it.state_words = mips.bricks.data_ptr(), mips.words.data_ptr()
    it.block_offset, it.active, it.n_active = (grid.block_offset.data_ptr(), grid.active.data_ptr(),
                                               grid.n_active_dev.data_ptr())
    it.n_dir = int(dirs_dev.shape[0])
    it.dirs, it.weights = dirs_dev.data_ptr(), weights_dev.data_ptr()
    b = [] if band is None else list(band)
    it.n_band = -1 if band is None else len(b)
    for q, v in enumerate(b[:4]):
        it.band[q] = float(v)
    it.i_bc = float(i_bc)
    it.J = J.data_ptr()
    return it


def batch_solve(ctx: Context, items, W: int, ctas: int = 0, queue: torch.Tensor | None = None,
                timing: bool = False):
    """One persistent launch over all atmospheres (``dex_batch_solve``).

    Returns ``(done_ns, start_ns)`` device tensors when ``timing`` (else ``(None, None)``)."""
    n = len(items)
    arr = (BatchItem * n)(*items)
    dev = torch.device("cuda", ctx.device)
    if queue is None:
        queue = torch.zeros(1, dtype=torch.int32, device=dev)
    done = torch.zeros(n, dtype=torch.int64, device=dev) if timing else None
    start = torch.zeros(1, dtype=torch.int64, device=dev) if timing else None
    ctx._rc(lib().dex_batch_solve(ctx.handle, n, arr, W, int(ctas), _ptr(queue), _ptr(done), _ptr(start)))
    return done, start


class BatchConfig(ctypes.Structure):
    """``dex_batch_config``: persistent grid size, probes per work item, items per
    queue claim, block-table staging (0 packed state words, 1 one word per block)."""
    _fields_ = [("ctas", ctypes.c_int), ("packet", ctypes.c_int), ("chunk", ctypes.c_int), ("staging", ctypes.c_int),
                ("occupancy", ctypes.c_int)]


def batch_solve_config(ctx: Context, items, W: int, ctas: int = 0, packet: int = 256, chunk: int = 1,
                       staging: int = 0, occupancy: int = 0, queue: torch.Tensor | None = None,
                       timing: bool = False):
    """``dex_batch_solve_config``: the batched solve with an explicit launch configuration."""
    n = len(items)
    arr = (BatchItem * n)(*items)
    dev = torch.device("cuda", ctx.device)
    if queue is None:
        queue = torch.zeros(1, dtype=torch.int32, device=dev)
    done = torch.zeros(n, dtype=torch.int64, device=dev) if timing else None
    start = torch.zeros(1, dtype=torch.int64, device=dev) if timing else None
    cfg = BatchConfig(int(ctas), int(packet), int(chunk), int(staging), int(occupancy))
    ctx._rc(lib().dex_batch_solve_config(ctx.handle, n, arr, W, ctypes.byref(cfg), _ptr(queue), _ptr(done),
                                         _ptr(start)))
    return done, start


def batch_solve_noalloc(ctx: Context, items, W: int, ctas: int = 0, done_ns: torch.Tensor | None = None,
                        start_ns: torch.Tensor | None = None):
    """``dex_batch_solve_noalloc``: the batched solve for callers that cannot allocate
    device memory when they solve (the work counter lives in the library's static
    scratch).  Outputs are the caller's; pass preallocated ``done_ns`` [n] and
    ``start_ns`` [1] int64 tensors to get completion times."""
    arr = (BatchItem * len(items))(*items)
    ctx._rc(lib().dex_batch_solve_noalloc(ctx.handle, len(items), arr, W, int(ctas), _ptr(done_ns), _ptr(start_ns)))


def measure_ex2_rate(ctx: Context) -> float:
    """Measured 2^x throughput of the special-function units (``dex_measure_ex2_rate``), per second."""
    v = ctypes.c_double(0.0)
    ctx._rc(lib().dex_measure_ex2_rate(ctx.handle, ctypes.byref(v)))
    return float(v.value)


def measure_fp32_rate(ctx: Context) -> float:
    """Measured FP32-pipe throughput on packed fused multiply-adds (``dex_measure_fp32_rate``),
    lane operations per second."""
    v = ctypes.c_double(0.0)
    ctx._rc(lib().dex_measure_fp32_rate(ctx.handle, ctypes.byref(v)))
    return float(v.value)


def selftest_wait_timeout(ctx: Context, polls: int = 1000):
    """Run the bounded-wait self-test (``dex_selftest_wait_timeout``); the next
    :meth:`Context.check` raises with DEX_ERR_TIMEOUT."""
    ctx._rc(lib().dex_selftest_wait_timeout(ctx.handle, int(polls)))


# ------------------------------------------------------ profile surrogate --

def mlp_param_count() -> int:
    return int(lib().dex_mlp_param_count())


def _samples(xau):
    if xau.dim() != 2 or xau.shape[1] != 3 or xau.dtype != torch.float32 or not xau.is_contiguous():
        raise ValueError("xau must be a contiguous [n][3] float32 tensor")
    return xau.shape[0]


def mlp_forward(ctx: Context, xau: torch.Tensor, params: torch.Tensor, out: torch.Tensor | None = None):
    """Predicted ln H(a, x - u) of the surrogate network (``dex_mlp_forward``)."""
    n = _samples(xau)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=xau.device)
    ctx._rc(lib().dex_mlp_forward(ctx.handle, n, _ptr(xau), _ptr(params), _ptr(out)))
    return out


def mlp_grad(ctx: Context, xau: torch.Tensor, target: torch.Tensor, params: torch.Tensor,
             grad: torch.Tensor | None = None, loss: torch.Tensor | None = None):
    """Mean squared error and its gradient (``dex_mlp_grad``); returns ``(grad, loss)``."""
    n = _samples(xau)
    if grad is None:
        grad = torch.empty(mlp_param_count(), dtype=torch.float32, device=xau.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=xau.device)
    ctx._rc(lib().dex_mlp_grad(ctx.handle, n, _ptr(xau), _ptr(target), _ptr(params), _ptr(grad), _ptr(loss)))
    return grad, loss


def mlp_adam(ctx: Context, params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8):
    """One Adam step in place on ``params`` (``dex_mlp_adam``)."""
    ctx._rc(lib().dex_mlp_adam(ctx.handle, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                               float(beta1), float(beta2), float(eps)))


def mlp_targets(ctx: Context, xau: torch.Tensor, out: torch.Tensor | None = None):
    """ln H(a, x - u) from the library's Voigt evaluation (``dex_mlp_targets``)."""
    n = _samples(xau)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=xau.device)
    ctx._rc(lib().dex_mlp_targets(ctx.handle, n, _ptr(xau), _ptr(out)))
    return out


def mlp_train(ctx: Context, xau: torch.Tensor, target: torch.Tensor, params: torch.Tensor, steps: int,
              batch: int, lr: float = 1e-3, lr_final: float | None = None, log_every: int = 0):
    """Minibatch Adam on the surrogate: each step is ``dex_mlp_grad`` on the next
    contiguous slice of the (caller-shuffled) samples, then ``dex_mlp_adam``.  The
    learning rate decays geometrically from ``lr`` to ``lr_final`` (default: constant).
    Returns the per-step losses logged every ``log_every`` steps (float list)."""
    n = _samples(xau)
    P = mlp_param_count()
    m = torch.zeros(P, dtype=torch.float32, device=xau.device)
    v = torch.zeros_like(m)
    grad = torch.empty_like(m)
    loss = torch.empty(1, dtype=torch.float32, device=xau.device)
    logged = []
    ratio = 1.0 if lr_final is None else (lr_final / lr) ** (1.0 / max(1, steps - 1))
    off = 0
    for k in range(steps):
        if off + batch > n:
            off = 0
        mlp_grad(ctx, xau[off:off + batch], target[off:off + batch], params, grad=grad, loss=loss)
        mlp_adam(ctx, params, grad, m, v, k + 1, lr * ratio ** k)
        off += batch
        if log_every and (k % log_every == 0 or k == steps - 1):
            logged.append(float(loss.item()))
    return logged


# ------------------------------------------------------------------- 3D --

BLOCK3 = 8


def _quadrature3(dirs, weights):
    d = _host_f32(dirs, (-1, 3))
    w = _host_f32(weights)
    if d.shape[0] != w.size:
        raise ValueError("dirs and weights differ in length")
    return d, w


def formal_solve_dense3(ctx: Context, nx: int, ny: int, nz: int, n_lambda: int, W: int, planes: torch.Tensor,
                        dirs, weights, probes: torch.Tensor | None = None, i_bc: float = 0.0,
                        want_intensity: bool = False, count_segments: bool = False,
                        J: torch.Tensor | None = None):
    """Plain full-resolution 3D solve (``dex_formal_solve_dense3``); ``planes`` from
    :func:`pack_planes` over the ``nx * ny * nz`` cells.  Returns ``(J, I, seg)`` as
    :func:`formal_solve_dense`."""
    d, w = _quadrature3(dirs, weights)
    dev = planes.device
    n_probe = nx * ny * nz if probes is None else int(probes.numel())
    n_probe_arg = -1 if probes is None else n_probe
    if J is None:
        J = torch.empty((n_lambda, n_probe), dtype=torch.float32, device=dev)
    I = torch.empty((n_lambda, d.shape[0], n_probe), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    ctx._rc(lib().dex_formal_solve_dense3(
        ctx.handle, nx, ny, nz, n_lambda, W, _ptr(planes), d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp),
        n_probe_arg, _ptr(probes) if n_probe_arg > 0 else None, float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


class SparseGrid3:
    """Block sparsity map and Morton layout (device tensors) of an nx x ny x nz grid."""

    def __init__(self, nx, ny, nz, block_offset, active, n_active):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nbx, self.nby, self.nbz = nx // BLOCK3, ny // BLOCK3, nz // BLOCK3
        self.block_offset = block_offset
        self.active = active
        self.n_active_dev = n_active

    @property
    def n_blocks(self):
        return self.nbx * self.nby * self.nbz

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    def n_active(self) -> int:
        return int(self.n_active_dev.item())


def grid3_build(ctx: Context, nx: int, ny: int, nz: int, eta: torch.Tensor, chi: torch.Tensor,
                out: SparseGrid3 | None = None):
    """3D sparsity map + Morton-ordered active blocks (``dex_grid3_build``)."""
    n_lambda = eta.shape[0]
    nb = (nx // BLOCK3) * (ny // BLOCK3) * (nz // BLOCK3)
    if out is None:
        dev = eta.device
        out = SparseGrid3(nx, ny, nz, torch.empty(nb, dtype=torch.int32, device=dev),
                          torch.zeros(nb, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.int32, device=dev))
    ctx._rc(lib().dex_grid3_build(ctx.handle, nx, ny, nz, n_lambda, _ptr(eta), _ptr(chi), _ptr(out.block_offset),
                                  _ptr(out.active), _ptr(out.n_active_dev)))
    return out


def state_words3(nx: int, ny: int, nz: int) -> int:
    return int(lib().dex_state_words3(nx, ny, nz))


def chain_voxels3(max_mip: int) -> int:
    return int(lib().dex_chain_voxels3(max_mip))


def mips3_build(ctx: Context, grid: SparseGrid3, eta, chi, W: int, max_mip: int, iod_eta: float, iod_chi: float,
                chi_ds_min: float = 0.25, log_mean: bool = False, level_cap: torch.Tensor | None = None,
                capacity: int | None = None, out: Mips | None = None, storage: int = STORE_F32):
    """3D MIP chains + VLM block levels of every wavelength batch (``dex_mips3_build``)."""
    n_lambda = eta.shape[0]
    cap = grid.n_blocks if capacity is None else int(capacity)
    n_batch = -(-n_lambda // W)
    if out is None:
        nf = int(lib().dex_brick3_floats(cap, n_lambda, W, max_mip, storage))
        bricks = torch.empty(max(nf, 4), dtype=torch.float32, device=eta.device)
        words = torch.empty((n_batch, state_words3(grid.nx, grid.ny, grid.nz)), dtype=torch.int64, device=eta.device)
        out = Mips(bricks, words, W, max_mip, n_lambda, cap, storage)
    p = VlmParams(float(iod_eta), float(iod_chi), float(chi_ds_min), int(max_mip), 1 if log_mean else 0,
                  int(out.storage))
    ctx._rc(lib().dex_mips3_build(ctx.handle, grid.nx, grid.ny, grid.nz, n_lambda, W, _ptr(eta), _ptr(chi),
                                  _ptr(grid.active), _ptr(grid.n_active_dev), cap, ctypes.byref(p), _ptr(level_cap),
                                  _ptr(out.bricks), _ptr(out.words)))
    return out


def formal_solve_hdda3(ctx: Context, grid: SparseGrid3, mips: Mips, dirs, weights, i_bc: float = 0.0,
                       want_intensity: bool = False, count_segments: bool = False, J: torch.Tensor | None = None,
                       band=None):
    """Accelerated 3D solve (``dex_formal_solve_hdda3``): dense ``J[n_lambda][nz*ny*nx]``
    (zero outside active blocks), optional I, optional integrated-segment count."""
    d, w = _quadrature3(dirs, weights)
    dev = mips.bricks.device
    n_cells = grid.n_cells
    if J is None:
        J = torch.empty((mips.n_lambda, n_cells), dtype=torch.float32, device=dev)
    I = torch.empty((mips.n_lambda, d.shape[0], n_cells), dtype=torch.float32, device=dev) if want_intensity else None
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    fp = ctypes.POINTER(ctypes.c_float)
    b = None if band is None else _host_f32(band).reshape(-1)
    ctx._rc(lib().dex_formal_solve_hdda3(
        ctx.handle, grid.nx, grid.ny, grid.nz, mips.n_lambda, mips.W, mips.max_mip, int(mips.storage),
        _ptr(mips.bricks), _ptr(mips.words), _ptr(grid.block_offset), _ptr(grid.active), _ptr(grid.n_active_dev),
        mips.capacity, d.shape[0], d.ctypes.data_as(fp), w.ctypes.data_as(fp), -1 if b is None else b.size,
        None if b is None else b.ctypes.data_as(fp), float(i_bc), _ptr(J), _ptr(I), _ptr(seg)))
    return J, I, seg


# ------------------------------------------------------ radiance cascades --

RC_LEVEL_CAP = (0, 0, 1, 2, 3, 4)


def rc_directions(n0: int, n_cascades: int) -> np.ndarray:
    """Directions of every cascade, concatenated: cascade i has n0 4^i directions
    theta_k = 2 pi (k + 1/2) / (n0 4^i) (float32 of the float64 cosine and sine)."""
    out = []
    for i in range(n_cascades):
        n = n0 * 4 ** i
        th = 2.0 * np.pi * (np.arange(n, dtype=np.float64) + 0.5) / n
        out.append(np.stack([np.cos(th), np.sin(th)], axis=1).astype(np.float32))
    return np.concatenate(out)


def rc_workspace_floats(nx: int, nz: int, n_lambda: int, W: int, n0: int) -> int:
    return int(lib().dex_rc_workspace_floats(nx, nz, n_lambda, W, n0))


def rc_solve(ctx: Context, grid: SparseGrid, mips: Mips, n_cascades: int = 6, n0: int = 4, t0: float = 1.5,
             level_cap=None, dirs=None, i_bc: float = 0.0, J: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, count_segments: bool = False):
    """Radiance-cascade formal solution over the sparse mipmapped grid (``dex_rc_solve``).

    ``level_cap``: per-cascade maximum MIP level (default the paper's [0, 0, 1, 2, 3, 4],
    truncated to ``n_cascades`` and clipped to the chains' top level); ``dirs``: every
    cascade's directions concatenated (default :func:`rc_directions`).  Returns
    ``(J, seg)`` with dense ``J[n_lambda][nz*nx]`` (zero outside non-empty blocks)."""
    dev = mips.bricks.device
    if level_cap is None:
        level_cap = [min(c, mips.max_mip) for c in (list(RC_LEVEL_CAP) + [4] * 8)[:n_cascades]]
    caps = (ctypes.c_int * n_cascades)(*[int(c) for c in level_cap])
    d = rc_directions(n0, n_cascades) if dirs is None else np.concatenate([np.asarray(x, np.float32).reshape(-1, 2)
                                                                             for x in dirs])
    d_dev = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
    n_cells = grid.nx * grid.nz
    if J is None:
        J = torch.empty((mips.n_lambda, n_cells), dtype=torch.float32, device=dev)
    if workspace is None:
        nf = rc_workspace_floats(grid.nx, grid.nz, mips.n_lambda, mips.W, n0)
        workspace = torch.empty(max(nf, 4), dtype=torch.float32, device=dev)
    seg = torch.zeros(1, dtype=torch.int64, device=dev) if count_segments else None
    ctx._rc(lib().dex_rc_solve(ctx.handle, grid.nx, grid.nz, mips.n_lambda, mips.W, mips.max_mip, int(mips.storage),
                               _ptr(mips.bricks), _ptr(mips.words), _ptr(grid.block_offset), mips.capacity,
                               n_cascades, n0, float(t0), caps, _ptr(d_dev), float(i_bc), _ptr(workspace), _ptr(J),
                               _ptr(seg)))
    return J, seg
