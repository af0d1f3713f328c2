"""Float64 oracle for the 3D adapted grid: sparsity map, Morton block layout,
variance-limited mipmapping over 2x2x2 groups and the expansion of the chosen
levels back onto MIP 0.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

The 3D form of ``mips.py`` (Section 2.1: MIPs over 2x2x2 voxels in 3D; Section
2.3: 8^3 blocks in 3D, one level per block, at most level 3 so that a block
reduces to one voxel).  The IoD test, the always-average rule, the log / linear
means and the batch-minimum level rule are those of the 2D oracle, applied to
the 8 children of a group.  Block k = (bz * nby + by) * nbx + bx; Morton order
interleaves (bx, by, bz) with x in bit 0, y in bit 1, z in bit 2 of each triple.
"""

from __future__ import annotations

import numpy as np

from .mips import _reduce


def block_empty(eta, chi, block: int = 8):
    """[nbz][nby][nbx] bool: every cell of the block has eta = chi = 0 at every wavelength."""
    eta = np.asarray(eta)
    chi = np.asarray(chi)
    if eta.ndim == 3:
        eta, chi = eta[None], chi[None]
    L, nz, ny, nx = eta.shape
    nbz, nby, nbx = nz // block, ny // block, nx // block
    nzb = (eta != 0) | (chi != 0)
    nzb = nzb.reshape(L, nbz, block, nby, block, nbx, block).any(axis=(0, 2, 4, 6))
    return ~nzb


def morton3(bx: int, by: int, bz: int) -> int:
    """Interleave the bits of (bx, by, bz): bit b of bx at 3b, of by at 3b + 1, of bz at 3b + 2."""
    code = 0
    for b in range(10):
        code |= ((bx >> b) & 1) << (3 * b)
        code |= ((by >> b) & 1) << (3 * b + 1)
        code |= ((bz >> b) & 1) << (3 * b + 2)
    return code


def block_layout(empty):
    """Morton-ordered active blocks: ``(active, offset)`` as in the 2D oracle."""
    empty = np.asarray(empty, dtype=bool)
    nbz, nby, nbx = empty.shape
    keyed = []
    for bz in range(nbz):
        for by in range(nby):
            for bx in range(nbx):
                if not empty[bz, by, bx]:
                    keyed.append((morton3(bx, by, bz), (bz * nby + by) * nbx + bx))
    keyed.sort()
    active = np.array([k for _, k in keyed], dtype=np.int32)
    offset = np.full(nbz * nby * nbx, -1, dtype=np.int32)
    for r, k in enumerate(active):
        offset[k] = r
    return active, offset.reshape(nbz, nby, nbx)


def _groups(a):
    L, Z, Y, X = a.shape
    g = a.reshape(L, Z // 2, 2, Y // 2, 2, X // 2, 2).transpose(0, 1, 3, 5, 2, 4, 6)
    return g.reshape(L, Z // 2, Y // 2, X // 2, 8)


def mip_chain(eta, chi, max_mip: int, thr_eta: float, thr_chi: float,
              chi_ds_min: float = 0.25, mean: str = "log", stats: bool = False):
    """Levels 0..max_mip of 3D (eta, chi) and the per-group pass flags of levels 1..max_mip.

    ``levels[m] = (eta_m, chi_m)`` of shape ``[L][nz >> m][ny >> m][nx >> m]``;
    ``passes[m - 1]`` the bool pass map of level m; with ``stats=True`` also per-level
    ``{"iod_eta", "iod_chi", "chi_ds"}``.
    """
    eta = np.asarray(eta, dtype=np.float64)
    chi = np.asarray(chi, dtype=np.float64)
    levels = [(eta, chi)]
    passes = []
    st = []
    for m in range(1, max_mip + 1):
        ds = float(2 ** m)
        ge, gc = _groups(levels[-1][0]), _groups(levels[-1][1])
        ve, iod_e = _reduce(ge, ds, mean)
        vc, iod_c = _reduce(gc, ds, mean)
        kds = gc.max(-1) * ds
        ok = ((iod_e < thr_eta) & (iod_c < thr_chi)) | (kds < chi_ds_min)
        levels.append((ve, vc))
        passes.append(ok)
        if stats:
            st.append({"iod_eta": iod_e, "iod_chi": iod_c, "chi_ds": kds})
    return (levels, passes, st) if stats else (levels, passes)


def block_levels(passes, empty, block: int, lambda_batch: int, level_cap=None, n_lambda: int | None = None):
    """[n_batch][nbz][nby][nbx] int: the largest level whose groups (and all finer ones)
    pass for every wavelength of the batch, capped by ``level_cap``; -1 for empty blocks."""
    empty = np.asarray(empty, dtype=bool)
    nbz, nby, nbx = empty.shape
    if not passes:
        n_batch = -(-int(n_lambda) // lambda_batch)
        return np.where(empty[None], -1, np.zeros((n_batch, nbz, nby, nbx), dtype=np.int32))
    L = passes[0].shape[0]
    n_batch = -(-L // lambda_batch)
    ok_all = np.ones((n_batch, nbz, nby, nbx), dtype=bool)
    level = np.zeros((n_batch, nbz, nby, nbx), dtype=np.int32)
    for m, ok in enumerate(passes, start=1):
        s = block >> m
        blk = ok.reshape(L, nbz, s, nby, s, nbx, s).all(axis=(2, 4, 6))
        per_batch = np.stack([blk[b * lambda_batch:(b + 1) * lambda_batch].all(axis=0) for b in range(n_batch)])
        ok_all &= per_batch
        level = np.where(ok_all, m, level)
    if level_cap is not None:
        level = np.minimum(level, np.maximum(np.asarray(level_cap), 0)[None])
    return np.where(empty[None], -1, level)


def expand(levels, level_map, lambda_batch: int):
    """MIP-0 grid where every cell takes the value of its block's chosen level (0 in empty blocks)."""
    eta0, chi0 = levels[0]
    L, nz, ny, nx = eta0.shape
    n_batch, nbz, nby, nbx = level_map.shape
    block = nz // nbz
    out_e = np.zeros_like(eta0)
    out_c = np.zeros_like(chi0)
    cell_level = np.repeat(np.repeat(np.repeat(level_map, block, axis=1), block, axis=2), block, axis=3)
    for l in range(L):
        lev = cell_level[l // lambda_batch]
        for m, (em, cm) in enumerate(levels):
            f = 2 ** m
            up_e = np.repeat(np.repeat(np.repeat(em[l], f, axis=0), f, axis=1), f, axis=2)
            up_c = np.repeat(np.repeat(np.repeat(cm[l], f, axis=0), f, axis=1), f, axis=2)
            sel = lev == m
            out_e[l][sel] = up_e[sel]
            out_c[l][sel] = up_c[sel]
    return out_e, out_c


def probes_of_blocks(empty, block: int = 8):
    """Cell indices (k * ny + j) * nx + i of every cell of every non-empty block (row-major)."""
    empty = np.asarray(empty, dtype=bool)
    keep = np.repeat(np.repeat(np.repeat(~empty, block, axis=0), block, axis=1), block, axis=2)
    return np.flatnonzero(keep.reshape(-1)).astype(np.int32)
