"""One walk per ray for each pair of wavelength batches b, n_batch - 1 - b on
the pair's minimum block levels, one thread carrying the pair's 16 wavelengths
(DEX_TRAVERSAL_PAIRED); an odd middle batch is solved alone.

In every block the walk uses the smaller of the pair's two VLM levels (Section
2.2), capped by the distance limits (Section 4.1); empty blocks stay empty.  So:

* against the float64 oracle solving on that level map (the plain solve on the
  grid expanded with it, or the distance-banded solve): 1e-5 relative on I and
  J, the accelerated bar;
* against the per-batch walk (k_solve_hdda_t) given state words that hold the
  pair's minimum for both batches: the same updates in the same order, so J and I
  are equal bit for bit -- for float32, bfloat16 and float16 bricks, with the
  early termination of opaque rays, ragged batches, one to nine batches and
  axis-parallel rays;
* configurations the paired walk does not support are refused with
  DEX_ERR_UNSUPPORTED.
"""

import numpy as np
import pytest

import synth
from levels_util import robust_level_mask
from oracle import lc, lines, mips as omips

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX, NZ, W = 128, 96, 8


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


def partners(n_batch, group=0):
    """Partner of every batch under the paired walk's rule: mirror-wise within
    consecutive groups of `group` batches (0: one group); a lone middle batch is
    its own partner."""
    g = n_batch if group <= 0 or group > n_batch else group
    out = np.arange(n_batch)
    for g0 in range(0, n_batch, g):
        size = min(g, n_batch - g0)
        for q in range(size):
            out[g0 + q] = g0 + size - 1 - q
    return out


def group_min(lev, group=0):
    """Per batch, the smaller of its own levels and its partner's (-1, empty,
    where either block is empty)."""
    return np.minimum(lev, lev[partners(lev.shape[0], group)])


def pack_states(lev, n_words):
    """Packed 3-bit block states (level + 1, 0 = empty), 21 per 64-bit word."""
    st = (lev + 1).astype(np.uint64).reshape(lev.shape[0], -1)
    k = np.arange(st.shape[1])
    out = np.zeros((st.shape[0], n_words), dtype=np.uint64)
    for b in range(st.shape[0]):
        np.bitwise_or.at(out[b], k // 21, st[b] << (3 * (k % 21)).astype(np.uint64))
    return out.view(np.int64)


def model(L, seed, shift, nx=NX, nz=NZ):
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=synth.SEED_BASE + seed)
    m["dlam"] = (m["dlam"] + shift).astype(m["dlam"].dtype)
    er, cr = lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])
    return m, er, cr


def build(ctx, m, thr, storage, nx=NX, nz=NZ):
    from paper_2511_08498_gb300 import api
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, 3, thr, thr, 0.25, log_mean=False, storage=storage)
    return grid, mp


def solve(ctx, grid, mp, dirs, w, band, mode, i_bc=0.0, group=0):
    from paper_2511_08498_gb300 import api
    ctx.set_traversal(mode)
    ctx.set_pair_group(group)
    try:
        J, I, seg = api.formal_solve_hdda(ctx, grid, mp, dirs, w, want_intensity=True, count_segments=True,
                                          band=band, i_bc=i_bc)
        ctx.check()
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
        ctx.set_pair_group(0)
    return J.cpu().numpy(), I.cpu().numpy(), int(seg.item())


# (wavelengths, seed, IoD threshold, distance limits, line-centre shift): 5 batches
# (groups of 4 and 1), 4.5 batches (ragged last batch), 3 batches, 4 batches, 9
# batches (groups of 4, 4 and 1)
CASES = [(40, 490, 1e-2, None, 5.0), (36, 491, 1.0, [5.3, 21.7, 60.1], 0.0), (24, 492, 1e-2, [2.2, 9.9], -3.5),
         (32, 493, 1e30, [6.0, 24.0, 96.0], 2.0), (72, 494, 1e-2, [6.0, 24.0, 96.0], 1.0)]


@pytest.mark.parametrize("L,seed,thr,band,shift", CASES)
def test_paired_walk_matches_oracle(ctx, L, seed, thr, band, shift):
    from paper_2511_08498_gb300 import api
    m, er, cr = model(L, seed, shift)
    dirs, w = synth.directions(12)
    grid, mp = build(ctx, m, thr, 0)
    J, I, seg = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED)
    glev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks).reshape(-1, NZ // 16, NX // 16)
    levels, passes, st = omips.mip_chain(er, cr, 3, thr, thr, 0.25, mean="linear", stats=True)
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W)
    assert robust_level_mask(st, lev, W, 16, 3, thr, thr, 0.25).all()
    np.testing.assert_array_equal(glev, lev)
    lev_c = group_min(lev)
    if thr < 1e29 and shift != 0.0:
        # a line centre off the middle of the wavelength grid gives the mirrored
        # batches different levels, so the pair's minimum is exercised
        assert not np.array_equal(lev_c, lev), "the pairs already have equal levels: the minimum is not exercised"
    probes = omips.probes_of_blocks(empty, 16)
    if band is None:
        e2, c2 = omips.expand(levels, lev_c, W)
        Jr, Ir = lc.formal_solve(e2, c2, dirs, w, probes=probes, want_intensity=True)
    else:
        Jr, Ir = lc.formal_solve_banded(levels, lev_c, 16, W, band, dirs, w, probes, want_intensity=True)
    assert rel(I[:, :, probes], Ir).max() < 1e-5
    assert rel(J[:, probes], Jr).max() < 1e-5
    zero = Jr == 0
    assert np.array_equal(J[:, probes][zero], Jr[zero])
    assert seg > 0


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("L,seed,thr,band,shift", [CASES[0], CASES[1], CASES[4]])
def test_paired_walk_equals_per_batch_walk_on_group_minimum(ctx, storage, L, seed, thr, band, shift):
    from paper_2511_08498_gb300 import api
    m, _, _ = model(L, seed, shift)
    dirs, w = synth.directions(12, offset=0.0)   # axis-parallel and diagonal rays included
    grid, mp = build(ctx, m, thr, storage)
    Jc, Ic, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED, i_bc=0.37)
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
    mp.words.copy_(torch.from_numpy(pack_states(group_min(lev), mp.words.shape[1])))
    Jp, Ip, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PER_BATCH, i_bc=0.37)
    assert np.array_equal(Ic, Ip)
    assert np.array_equal(Jc, Jp)


def test_paired_walk_thick_and_single_batch(ctx):
    """One batch (solved alone), then two (one pair); one direction and then 37; an
    opaque atmosphere whose rays all end early."""
    from paper_2511_08498_gb300 import api
    for L, n_dir in ((8, 1), (16, 37)):
        m, _, _ = model(L, 495, 0.0)
        m["chi_c"] = (m["chi_c"] * 1e4).astype(m["chi_c"].dtype)
        grid, mp = build(ctx, m, 1e-2, 0)
        dirs, w = synth.directions(n_dir)
        Jc, Ic, _ = solve(ctx, grid, mp, dirs, w, [6.0, 24.0, 96.0], api.TRAVERSAL_PAIRED)
        lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
        mp.words.copy_(torch.from_numpy(pack_states(group_min(lev), mp.words.shape[1])))
        Jp, Ip, _ = solve(ctx, grid, mp, dirs, w, [6.0, 24.0, 96.0], api.TRAVERSAL_PER_BATCH)
        assert np.array_equal(Ic, Ip)
        assert np.array_equal(Jc, Jp)


def test_paired_walk_unsupported_configurations(ctx):
    from paper_2511_08498_gb300 import _native, api
    m, _, _ = model(16, 496, 0.0)
    dirs, w = synth.directions(4)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    grid = api.grid_build(ctx, NX, NZ, eg, cg)
    mp4 = api.mips_build(ctx, grid, eg, cg, 4, 3, 1e-2, 1e-2, 0.25)
    ctx.set_traversal(api.TRAVERSAL_PAIRED)
    try:
        with pytest.raises(api.DexError) as ex:
            api.formal_solve_hdda(ctx, grid, mp4, dirs, w)
        assert ex.value.code == 16   # DEX_ERR_UNSUPPORTED: W = 4
        mp8 = api.mips_build(ctx, grid, eg, cg, 8, 3, 1e-2, 1e-2, 0.25, storage=1)
        ctx.set_own_cell(False)
        with pytest.raises(api.DexError) as ex:
            api.formal_solve_hdda(ctx, grid, mp8, dirs, w)
        assert ex.value.code == 16   # own-cell emission left out: float32 bricks only
    finally:
        ctx.set_own_cell(True)
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
    assert _native.lib().dex_ctx_set_traversal(ctx.handle, 3) == 1   # DEX_ERR_ARG
    assert _native.lib().dex_ctx_set_pair_group(ctx.handle, -1) == 1  # DEX_ERR_ARG


def test_pair_rule():
    assert list(partners(5)) == [4, 3, 2, 1, 0]
    assert list(partners(5, 2)) == [1, 0, 3, 2, 4]
    assert list(partners(12, 5)) == [4, 3, 2, 1, 0, 9, 8, 7, 6, 5, 11, 10]


# (wavelengths, pair group): 5 batches in groups of 2 (pairs 0-1, 2-3, batch 4
# alone) and of 3 (0-2, 3-4, batch 1 alone); 12 batches in groups of 5, the
# layout of two 40-sample lines and a 16-sample continuum
@pytest.mark.parametrize("L,group", [(40, 2), (40, 3), (96, 5)])
def test_paired_walk_groups(ctx, L, group):
    from paper_2511_08498_gb300 import api
    m, er, cr = model(L, 497, 3.0)
    dirs, w = synth.directions(8, offset=0.0)
    band = [6.0, 24.0, 96.0]
    grid, mp = build(ctx, m, 1e-2, 0)
    Jc, Ic, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED, i_bc=0.11, group=group)
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
    if L == 40:
        # against the float64 oracle on the pair-minimum map of this grouping
        levels, passes, st = omips.mip_chain(er, cr, 3, 1e-2, 1e-2, 0.25, mean="linear", stats=True)
        empty = omips.block_empty(er, cr, 16)
        lev_r = omips.block_levels(passes, empty, 16, W)
        assert robust_level_mask(st, lev_r, W, 16, 3, 1e-2, 1e-2, 0.25).all()
        assert np.array_equal(lev.reshape(lev_r.shape), lev_r)
        lev_c = group_min(lev_r, group)
        assert not np.array_equal(lev_c, lev_r)
        probes = omips.probes_of_blocks(empty, 16)
        Jr, Ir = lc.formal_solve_banded(levels, lev_c, 16, W, band, dirs, w, probes, i_bc=0.11, want_intensity=True)
        assert rel(Ic[:, :, probes], Ir).max() < 1e-5
        assert rel(Jc[:, probes], Jr).max() < 1e-5
    # bit for bit against the per-batch walk on the same map
    mp.words.copy_(torch.from_numpy(pack_states(group_min(lev, group), mp.words.shape[1])))
    Jp, Ip, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PER_BATCH, i_bc=0.11)
    assert np.array_equal(Ic, Ip)
    assert np.array_equal(Jc, Jp)


def test_paired_walk_without_own_cell(ctx):
    """The own-cell emission left out (the MALI solves' Jext): the paired walk
    equals the per-batch walk on the pair-minimum map bit for bit, pairs within
    groups of two and a lone batch included."""
    from paper_2511_08498_gb300 import api
    m, _, _ = model(40, 498, 2.0)
    dirs, w = synth.directions(8)
    band = [6.0, 24.0, 96.0]
    grid, mp = build(ctx, m, 1e-2, 0)
    ctx.set_own_cell(False)
    try:
        Jc, Ic, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PAIRED, group=2)
        lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
        mp.words.copy_(torch.from_numpy(pack_states(group_min(lev, 2), mp.words.shape[1])))
        Jp, Ip, _ = solve(ctx, grid, mp, dirs, w, band, api.TRAVERSAL_PER_BATCH)
    finally:
        ctx.set_own_cell(True)
    assert np.array_equal(Ic, Ip)
    assert np.array_equal(Jc, Jp)


def _banded_grid(nx, nz, L, rows):
    """eta, chi on device: a smooth medium in the bottom `rows` cells, the same at
    every wavelength (so every batch takes the same levels), empty above."""
    x = torch.arange(nx, device="cuda", dtype=torch.float32)[None, :] + 0.5
    z = torch.arange(rows, device="cuda", dtype=torch.float32)[:, None] + 0.5
    chi_b = 0.05 * (1.5 + torch.sin(2 * np.pi * x / 300.0)) * torch.exp(-z / 20.0)
    eta_b = chi_b * (1.0 + 0.5 * torch.cos(2 * np.pi * x / 170.0))
    chi = torch.zeros((L, nz, nx), device="cuda")
    eta = torch.zeros_like(chi)
    chi[:, :rows, :] = chi_b
    eta[:, :rows, :] = eta_b
    return eta.reshape(L, -1), chi.reshape(L, -1)


def test_paired_walk_above_the_per_batch_staged_table(ctx):
    """The paired walk stages one word per block for grids of up to 16384 blocks (the
    per-batch walk only up to 8192, reading the packed words beyond): on a 2560 x 1024
    grid (10240 blocks) the paired walk equals the per-batch walk bit for bit."""
    from paper_2511_08498_gb300 import api
    nx, nz, L = 2560, 1024, 16
    eg, cg = _banded_grid(nx, nz, L, 64)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    assert 8192 < grid.n_blocks <= 16384
    mp = api.mips_build(ctx, grid, eg, cg, W, 3, 1e-2, 1e-2, 0.25, log_mean=False, capacity=grid.n_active())
    dirs, w = synth.directions(8)
    band = [6.0, 24.0, 96.0]
    Jb, _, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w, band=band)
    ctx.set_traversal(api.TRAVERSAL_PAIRED)
    try:
        Jp, _, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w, band=band)
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
    ctx.check()
    assert float(Jb.abs().max()) > 0.0
    assert torch.equal(Jb, Jp)


def test_paired_walk_refuses_grids_above_16384_blocks(ctx):
    from paper_2511_08498_gb300 import api
    nx, nz, L = 4096, 1040, 8
    eg, cg = _banded_grid(nx, nz, L, 16)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    assert grid.n_blocks > 16384
    mp = api.mips_build(ctx, grid, eg, cg, W, 3, 1e-2, 1e-2, 0.25, log_mean=False, capacity=grid.n_active())
    dirs, w = synth.directions(4)
    ctx.set_traversal(api.TRAVERSAL_PAIRED)
    try:
        with pytest.raises(api.DexError) as ex:
            api.formal_solve_hdda(ctx, grid, mp, dirs, w)
        assert ex.value.code == 16   # DEX_ERR_UNSUPPORTED
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
    J, _, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w)   # the per-batch walk takes it
    ctx.check()
