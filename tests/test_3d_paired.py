"""3D accelerated solve with one walk per mirror pair of wavelength batches
(DEX_TRAVERSAL_PAIRED; 8^3 blocks, levels 0..3) on the GPU.

The walk uses, in every block, the smaller of the levels of batches b and
n_batch - 1 - b (Section 2.2), capped by the distance limits (Section 4.1); an
odd middle batch is solved alone.  So:

* against the float64 3D oracle solving on that pair-minimum level map (the
  distance-banded solve): 1e-5 relative on I and J, with the line centre moved
  off the middle of the wavelength grid so that the mirrored batches take
  different levels;
* against the per-batch 3D walk given state words that hold the pair minimum
  for both batches: bit for bit, for float32, bfloat16 and float16 bricks, and
  with the batches paired within groups of two.
"""

import numpy as np
import pytest

import synth
from levels_util import robust_level_mask3
from oracle import lc3, lines, mips3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-30)


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    c = api.Context(0)
    yield c
    c.set_traversal(api.TRAVERSAL_PER_BATCH)


def pair_min(lev, group=0):
    """Per batch, the smaller of its own levels and its partner's: mirror-wise
    within consecutive groups of `group` batches (0: one group)."""
    n = lev.shape[0]
    g = n if group <= 0 or group > n else group
    part = np.arange(n)
    for g0 in range(0, n, g):
        size = min(g, n - g0)
        part[g0:g0 + size] = g0 + size - 1 - np.arange(size)
    return np.minimum(lev, lev[part])


def pack_states(lev, n_words):
    """Packed 3-bit block states (level + 1, 0 = empty), 21 per 64-bit word."""
    st = (lev + 1).astype(np.uint64).reshape(lev.shape[0], -1)
    k = np.arange(st.shape[1])
    out = np.zeros((st.shape[0], n_words), dtype=np.uint64)
    for b in range(st.shape[0]):
        np.bitwise_or.at(out[b], k // 21, st[b] << (3 * (k % 21)).astype(np.uint64))
    return out.view(np.int64)


def line3(ctx, nx, ny, nz, L, seed, shift):
    from paper_2511_08498_gb300 import api
    m = synth.sparse_line_atmosphere3(nx, ny, nz, n_lambda=L, seed=seed)
    m["dlam"] = (m["dlam"] + shift).astype(m["dlam"].dtype)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    er, cr = lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])
    # the oracle takes the GPU's float32 MIP-0 values (line synthesis is pinned separately)
    e32 = eg.cpu().numpy().reshape(er.shape).astype(np.float64)
    c32 = cg.cpu().numpy().reshape(cr.shape).astype(np.float64)
    assert np.allclose(e32, er, rtol=2e-6, atol=0) and np.allclose(c32, cr, rtol=2e-6, atol=0)
    return eg, cg, e32, c32


def solve(ctx, grid, mp, dirs, w, band, mode, group=0):
    from paper_2511_08498_gb300 import api
    ctx.set_traversal(mode)
    ctx.set_pair_group(group)
    try:
        J, I, seg = api.formal_solve_hdda3(ctx, grid, mp, dirs, w, band=band, want_intensity=True, i_bc=0.21)
        ctx.check()
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
        ctx.set_pair_group(0)
    return J.cpu().numpy(), I.cpu().numpy()


@pytest.mark.parametrize("L,thr,band,shift", [(40, 0.1, [4.0, 12.0, 24.0], 3.0), (24, 1e30, [3.0, 9.0, 20.0], -2.0)])
def test_paired_3d_walk_matches_oracle(ctx, L, thr, band, shift):
    from paper_2511_08498_gb300 import api
    nx, ny, nz = 48, 40, 32
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 197, shift)
    dirs, w = synth.directions3(6, 3)
    grid = api.grid3_build(ctx, nx, ny, nz, eg, cg)
    mp = api.mips3_build(ctx, grid, eg, cg, 8, 3, thr, thr, 0.25)
    J, I = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED)
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks).reshape(-1, nz // 8, ny // 8, nx // 8)
    levels, passes, st = mips3.mip_chain(er, cr, 3, thr, thr, 0.25, mean="linear", stats=True)
    empty = mips3.block_empty(er, cr, 8)
    lev_r = mips3.block_levels(passes, empty, 8, 8)
    assert robust_level_mask3(st, lev_r, 8, 3, thr, thr, 0.25).all()
    assert np.array_equal(lev, lev_r)
    lev_c = pair_min(lev_r)
    if thr < 1e29:
        assert not np.array_equal(lev_c, lev_r), "the pairs already have equal levels: the minimum is not exercised"
    probes = mips3.probes_of_blocks(empty, 8)
    Jr, Ir = lc3.formal_solve_banded(levels, lev_c, 8, 8, band, dirs, w, probes, i_bc=0.21, want_intensity=True)
    assert rel(I[:, :, probes], Ir).max() < 1e-5
    assert rel(J[:, probes], Jr).max() < 1e-5


@pytest.mark.parametrize("storage,group", [(0, 0), (1, 0), (2, 0), (0, 2)])
def test_paired_3d_walk_equals_per_batch_walk_on_pair_minimum(ctx, storage, group):
    from paper_2511_08498_gb300 import api
    nx, ny, nz, L = 40, 32, 48, 36                      # 4.5 batches: pairs (0, 4), (1, 3), batch 2 alone
    eg, cg, _, _ = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 198, 4.0)
    dirs, w = synth.directions3(4, 2, offset=0.0)       # axis-parallel rays included
    grid = api.grid3_build(ctx, nx, ny, nz, eg, cg)
    mp = api.mips3_build(ctx, grid, eg, cg, 8, 3, 0.1, 0.1, 0.25, storage=storage)
    band = [4.0, 12.0, 24.0]
    Jc, Ic = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED, group=group)
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
    mp.words.copy_(torch.from_numpy(pack_states(pair_min(lev, group), mp.words.shape[1])))
    Jp, Ip = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PER_BATCH)
    assert np.array_equal(Ic, Ip)
    assert np.array_equal(Jc, Jp)
