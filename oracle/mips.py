"""Float64 oracle for the adapted grid: sparsity map, block layout, variance-limited
mipmapping (VLM) and the expansion of the chosen MIP levels back onto MIP 0.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

Readings of the paper taken here (each listed in the design notes):

* Section 2.1 / Fig. 2: MIP level m has voxels of side 2^m built from the 2x2
  children of level m-1.  The chain is built per wavelength.
* Section 2.2, Eq. IoD: IoD[X] = |Var[X] / Mean[X]| over the 4 children, with
  X = ln(eta Ds) and X = ln(chi Ds), Ds = 2^m the side of the voxel being
  formed, Var the population variance.  A group passes when both IoDs are below
  their thresholds, or (always-average rule) when chi Ds < chi_ds_min, taken as
  the largest child chi times Ds.
* Averaging: log-space (geometric) mean of the children, the default; the
  paper's Fig. 2 box filter (arithmetic mean) is the ``"linear"`` option.  A
  group whose children mix zeros and non-zeros has no log mean: its IoD is
  infinite (it can only pass through the always-average rule) and its value is
  the arithmetic mean.  An all-zero group has value 0 and IoD 0.
* Section 2.3.1: a block stores the largest level m (<= max_mip) such that every
  group at every level 1..m inside it passes, for every wavelength of a
  wavelength batch (Section 4.1: one level structure per batch of consecutive
  wavelengths).  Empty blocks (eta = chi = 0 for every cell and wavelength) get
  level -1.  Block states are packed 3 bits each (0 = empty, m + 1 = level m),
  21 states per 64-bit word, block k in word k // 21 at bit 3 (k % 21), with
  k = bz * nbx + bx.
* Section 2.3.1: active blocks are laid out along the Morton Z-order curve of
  their (bx, bz) block coordinates (bit-interleaved, x in the even bits); an
  offset table maps each block to its rank in that order, -1 when empty.
"""

from __future__ import annotations

import numpy as np


def block_empty(eta, chi, block: int):
    """[nbz][nbx] bool: every cell of the block has eta = chi = 0 at every wavelength."""
    eta = np.asarray(eta)
    chi = np.asarray(chi)
    if eta.ndim == 2:
        eta, chi = eta[None], chi[None]
    L, nz, nx = eta.shape
    nbz, nbx = nz // block, nx // block
    nz_b = (eta != 0) | (chi != 0)
    nz_b = nz_b.reshape(L, nbz, block, nbx, block).any(axis=(0, 2, 4))
    return ~nz_b


def morton2(bx: int, bz: int) -> int:
    """Interleave the bits of (bx, bz): bx in the even bits, bz in the odd bits."""
    code = 0
    for b in range(16):
        code |= ((bx >> b) & 1) << (2 * b)
        code |= ((bz >> b) & 1) << (2 * b + 1)
    return code


def block_layout(empty):
    """Morton-ordered active blocks.

    Returns ``(active, offset)``: ``active[r]`` is the row-major block index
    ``bz * nbx + bx`` of the r-th active block along the Z-order curve and
    ``offset[bz][bx]`` its rank (-1 for empty blocks).
    """
    empty = np.asarray(empty, dtype=bool)
    nbz, nbx = empty.shape
    keyed = []
    for bz in range(nbz):
        for bx in range(nbx):
            if not empty[bz, bx]:
                keyed.append((morton2(bx, bz), bz * nbx + bx))
    keyed.sort()
    active = np.array([k for _, k in keyed], dtype=np.int32)
    offset = np.full((nbz, nbx), -1, dtype=np.int32)
    for r, k in enumerate(active):
        offset[k // nbx, k % nbx] = r
    return active, offset


def _groups(a):
    L, Z, X = a.shape
    return a.reshape(L, Z // 2, 2, X // 2, 2).transpose(0, 1, 3, 2, 4).reshape(L, Z // 2, X // 2, 4)


def _reduce(g, ds: float, mean: str):
    """Value and IoD of the 2x2 groups g[..., 4] at voxel side ds."""
    pos = g > 0
    allpos = pos.all(-1)
    allzero = (g == 0).all(-1)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        X = np.log(np.where(pos, g * ds, 1.0))
        mu = X.mean(-1)
        var = ((X - mu[..., None]) ** 2).mean(-1)
        iod = np.abs(var / mu)
    iod = np.where(var == 0.0, 0.0, iod)
    iod = np.where(allpos, iod, np.where(allzero, 0.0, np.inf))
    lin = g.mean(-1)
    if mean == "log":
        with np.errstate(divide="ignore"):
            geo = np.exp(np.log(np.where(pos, g, 1.0)).mean(-1))
        val = np.where(allpos, geo, np.where(allzero, 0.0, lin))
    elif mean == "linear":
        val = lin
    else:
        raise ValueError(mean)
    return val, iod


def mip_chain(eta, chi, max_mip: int, thr_eta: float, thr_chi: float,
              chi_ds_min: float = 0.25, mean: str = "log", stats: bool = False):
    """Levels 0..max_mip of (eta, chi) and the per-group pass flags of levels 1..max_mip.

    Returns ``(levels, passes)``: ``levels[m] = (eta_m, chi_m)`` of shape
    ``[L][nz >> m][nx >> m]``; ``passes[m - 1]`` is the bool pass map of level m.
    With ``stats=True`` also a list of per-level dicts ``{"iod_eta", "iod_chi",
    "chi_ds"}`` (the quantities each group's decision compares with its thresholds).
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
    """[n_batch][nbz][nbx] int: the largest level whose groups (and all finer ones) pass
    for every wavelength of the batch, at most ``level_cap[bz][bx]`` when given; -1 for
    empty blocks.  With no level above 0 (``passes == []``) every block is at level 0,
    which needs ``n_lambda``."""
    empty = np.asarray(empty, dtype=bool)
    nbz, nbx = empty.shape
    if not passes:
        n_batch = -(-int(n_lambda) // lambda_batch)
        return np.where(empty[None], -1, np.zeros((n_batch, nbz, nbx), dtype=np.int32))
    L = passes[0].shape[0]
    n_batch = -(-L // lambda_batch)
    ok_all = np.ones((n_batch, nbz, nbx), dtype=bool)
    level = np.zeros((n_batch, nbz, nbx), dtype=np.int32)
    for m, ok in enumerate(passes, start=1):
        side = block >> m
        blk = ok.reshape(L, nbz, side, nbx, side).all(axis=(2, 4))  # [L][nbz][nbx]
        per_batch = np.stack([blk[b * lambda_batch:(b + 1) * lambda_batch].all(axis=0)
                              for b in range(n_batch)])
        ok_all &= per_batch
        level = np.where(ok_all, m, level)
    if level_cap is not None:
        level = np.minimum(level, np.maximum(np.asarray(level_cap), 0)[None])
    level = np.where(empty[None], -1, level)
    return level


def expand(levels, level_map, lambda_batch: int):
    """MIP-0 grid where every cell takes the value of its block's chosen level.

    level_map: ``[n_batch][nbz][nbx]``.  Returns float64 ``(eta, chi)`` of shape
    ``[L][nz][nx]``; cells of empty blocks are 0.
    """
    eta0, chi0 = levels[0]
    L, nz, nx = eta0.shape
    n_batch, nbz, nbx = level_map.shape
    block = nz // nbz
    out_e = np.zeros_like(eta0)
    out_c = np.zeros_like(chi0)
    cell_level = np.repeat(np.repeat(level_map, block, axis=1), block, axis=2)  # [n_batch][nz][nx]
    for l in range(L):
        lev = cell_level[l // lambda_batch]
        for m, (em, cm) in enumerate(levels):
            f = 2 ** m
            up_e = np.repeat(np.repeat(em[l], f, axis=0), f, axis=1)
            up_c = np.repeat(np.repeat(cm[l], f, axis=0), f, axis=1)
            sel = lev == m
            out_e[l][sel] = up_e[sel]
            out_c[l][sel] = up_c[sel]
    return out_e, out_c


def pack_states(level_map_2d, bits: int = 3):
    """Pack block states (level + 1, 0 = empty) of one level map into uint64 words."""
    lev = np.asarray(level_map_2d).reshape(-1)
    per = 64 // bits
    n_words = -(-lev.size // per)
    words = np.zeros(n_words, dtype=np.uint64)
    for k, v in enumerate(lev):
        state = int(v) + 1
        if state < 0 or state >= (1 << bits):
            raise ValueError("state does not fit")
        words[k // per] |= np.uint64(state << (bits * (k % per)))
    return words


def unpack_states(words, n_blocks: int, bits: int = 3):
    per = 64 // bits
    out = np.zeros(n_blocks, dtype=np.int32)
    for k in range(n_blocks):
        out[k] = int((int(words[k // per]) >> (bits * (k % per))) & ((1 << bits) - 1)) - 1
    return out


def probes_of_blocks(empty, block: int):
    """Cell indices j * nx + i of every cell in every non-empty block (row-major order)."""
    empty = np.asarray(empty, dtype=bool)
    nbz, nbx = empty.shape
    keep = np.repeat(np.repeat(~empty, block, axis=0), block, axis=1)
    return np.flatnonzero(keep.reshape(-1)).astype(np.int32)
