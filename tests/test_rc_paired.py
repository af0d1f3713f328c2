"""Radiance cascades with one walk per pair of wavelength batches
(DEX_TRAVERSAL_PAIRED): every cascade interval walks once for a pair of batches
on the smaller of their two levels (capped by the cascade's level cap), lone
batches alone.  With state words that hold the pair minimum for both batches,
the per-batch cascades trace the same voxels with the same lengths and merge
the same way, so J must equal theirs bit for bit -- for F32, BF16 and F16
bricks, mirror pairs and pairs within groups of two, with a boundary intensity.
The per-batch cascades are checked against the float64 cascade oracle in
tests/test_rc_parity.py."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def partners(n_batch, group=0):
    g = n_batch if group <= 0 or group > n_batch else group
    out = np.arange(n_batch)
    for g0 in range(0, n_batch, g):
        size = min(g, n_batch - g0)
        out[g0:g0 + size] = g0 + size - 1 - np.arange(size)
    return out


def pack_states(lev, n_words):
    st = (lev + 1).astype(np.uint64).reshape(lev.shape[0], -1)
    k = np.arange(st.shape[1])
    out = np.zeros((st.shape[0], n_words), dtype=np.uint64)
    for b in range(st.shape[0]):
        np.bitwise_or.at(out[b], k // 21, st[b] << (3 * (k % 21)).astype(np.uint64))
    return out.view(np.int64)


@pytest.mark.parametrize("storage,group,L", [(0, 0, 40), (1, 0, 32), (2, 2, 40), (0, 2, 24)])
def test_paired_cascades_equal_per_batch_cascades_on_pair_minimum(storage, group, L):
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    nx, nz, C, n0 = 128, 96, 5, 4
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=synth.SEED_BASE + 530 + L)
    m["dlam"] = (m["dlam"] + 3.0).astype(m["dlam"].dtype)   # mirrored batches with different levels
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, 8, 3, 1e-2, 1e-2, 0.25, storage=storage)
    caps = [0, 0, 1, 2, 3]
    dirs = synth.rc_directions(n0, C)
    ctx.set_traversal(api.TRAVERSAL_PAIRED)
    ctx.set_pair_group(group)
    try:
        Jc, _ = api.rc_solve(ctx, grid, mp, n_cascades=C, n0=n0, level_cap=caps, dirs=dirs, i_bc=0.3)
        ctx.check()
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
        ctx.set_pair_group(0)
    Jc = Jc.cpu().numpy()
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
    lev_c = np.minimum(lev, lev[partners(lev.shape[0], group)])
    if group == 0:
        # the line centre sits off the middle of the wavelength grid: mirrored
        # batches take different levels and the pair minimum is exercised
        assert not np.array_equal(lev_c, lev)
    mp.words.copy_(torch.from_numpy(pack_states(lev_c, mp.words.shape[1])))
    Jp, _ = api.rc_solve(ctx, grid, mp, n_cascades=C, n0=n0, level_cap=caps, dirs=dirs, i_bc=0.3)
    ctx.check()
    assert np.array_equal(Jc, Jp.cpu().numpy())
