"""Sparse block grid, VLM MIP build and HDDA solve on the GPU vs the float64 oracle.

* line synthesis: within 2e-6 relative (float32 arithmetic, a handful of roundings);
* block sparsity map and Morton layout: bit-exact;
* block levels: exact wherever the oracle's decision is not within 1e-4 (relative)
  of a threshold -- the GPU decides in float32, the oracle in float64 -- and the
  tested inputs are checked to have no such ambiguous block;
* MIP values of the selected levels: within 1e-5 relative;
* HDDA intensities and J: within 1e-5 relative of the plain oracle run on the
  grid where each cell takes its block's selected-level value (the composition
  of piecewise-constant segments is exact, so HDDA must reproduce it).
"""

import numpy as np
import pytest

import synth
from levels_util import robust_level_mask
from oracle import lc, lines, mips as omips

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5


def assert_rel(gpu, ref, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    zero = ref == 0
    assert np.array_equal(gpu[zero], ref[zero]), f"{what}: exact zeros differ ({np.count_nonzero(gpu[zero])})"
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-30)
    worst = np.unravel_index(np.argmax(rel), rel.shape)
    assert rel.max() <= rtol, f"{what}: max rel err {rel.max():.3e} at {worst}: gpu {gpu[worst]} ref {ref[worst]}"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


def line_model(nx, nz, n_lambda, seed):
    return synth.sparse_line_atmosphere(nx, nz, n_lambda=n_lambda, seed=seed)


def gpu_line_eta_chi(ctx, m):
    from paper_2511_08498_gb300 import api
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    return api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])


def oracle_line_eta_chi(m):
    return lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])


def gpu_pipeline(ctx, nx, nz, eta, chi, W, max_mip, te, tc, cm=0.25, log_mean=True, level_cap=None,
                 dirs=None, w=None, i_bc=0.0, want_I=True):
    from paper_2511_08498_gb300 import api
    grid = api.grid_build(ctx, nx, nz, eta, chi)
    cap_t = None if level_cap is None else torch.from_numpy(np.asarray(level_cap, np.int8).reshape(-1)).cuda()
    mp = api.mips_build(ctx, grid, eta, chi, W, max_mip, te, tc, cm, log_mean=log_mean, level_cap=cap_t)
    J, I, seg = api.formal_solve_hdda(ctx, grid, mp, dirs, w, i_bc=i_bc, want_intensity=want_I, count_segments=True)
    ctx.check()
    return grid, mp, J, I, seg


def oracle_pipeline(eta, chi, W, max_mip, te, tc, cm=0.25, mean="log", level_cap=None, dirs=None, w=None,
                    i_bc=0.0, stats=False):
    L, nz, nx = eta.shape
    empty = omips.block_empty(eta, chi, 16)
    res = omips.mip_chain(eta, chi, max_mip, te, tc, cm, mean=mean, stats=True)
    levels, passes, st = res
    lev = omips.block_levels(passes, empty, 16, W, level_cap=level_cap, n_lambda=L)
    e2, c2 = omips.expand(levels, lev, W)
    probes = omips.probes_of_blocks(empty, 16)
    J, I = lc.formal_solve(e2, c2, dirs, w, probes=probes, i_bc=i_bc, want_intensity=True)
    return dict(empty=empty, levels=levels, lev=lev, stats=st, probes=probes, J=J, I=I)


# ------------------------------------------------------------------ tests --

def test_static_line_synthesis(ctx):
    m = line_model(128, 96, 16, synth.SEED_BASE + 400)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    assert_rel(cg.cpu().numpy(), cr.reshape(16, -1), 2e-6, "chi")
    assert_rel(eg.cpu().numpy(), er.reshape(16, -1), 2e-6, "eta")


def test_grid_build_layout_bit_exact(ctx):
    from paper_2511_08498_gb300 import api
    for (nx, nz, seed) in [(256, 128, 401), (128, 192, 402), (16, 16, 403)]:
        m = line_model(nx, nz, 8, synth.SEED_BASE + seed)
        eg, cg = gpu_line_eta_chi(ctx, m)
        grid = api.grid_build(ctx, nx, nz, eg, cg)
        er, cr = oracle_line_eta_chi(m)
        empty = omips.block_empty(er, cr, 16)
        active, offset = omips.block_layout(empty)
        assert grid.n_active() == active.size
        np.testing.assert_array_equal(grid.block_offset.cpu().numpy(), offset.reshape(-1))
        np.testing.assert_array_equal(grid.active.cpu().numpy()[:active.size], active)


@pytest.mark.parametrize("max_mip,te,log_mean", [(3, 1e-2, True), (3, 1e-3, True), (2, 1.0, True),
                                                 (3, 1e-2, False), (4, 1.0, True)])
def test_vlm_levels_and_mip_values(ctx, max_mip, te, log_mean):
    from paper_2511_08498_gb300 import api
    nx, nz, L, W = 128, 96, 16, 8
    m = line_model(nx, nz, L, synth.SEED_BASE + 410)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, max_mip, te, te, 0.25, log_mean=log_mean)
    ctx.check()
    mean = "log" if log_mean else "linear"
    levels, passes, st = omips.mip_chain(er, cr, max_mip, te, te, 0.25, mean=mean, stats=True)
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W)
    nbz, nbx = empty.shape
    glev = api.unpack_states(mp.words.cpu().numpy(), nbz * nbx).reshape(lev.shape)
    robust = robust_level_mask(st, lev, W, 16, max_mip, te, te, 0.25)
    assert robust.mean() > 0.97, f"too many ambiguous blocks: {1 - robust.mean():.3f}"
    np.testing.assert_array_equal(glev[robust], lev[robust])
    # the MIP values of every level of every active block
    active, _ = omips.block_layout(empty)
    chain = api.chain_voxels(max_mip)
    bricks = mp.bricks.cpu().numpy()[: (L // W) * grid.n_blocks * chain * 2 * W]
    bricks = bricks.reshape(L // W, grid.n_blocks, chain, 2 * W)
    off = [341 - (341 >> (2 * k)) for k in range(5)]
    for r, blk in enumerate(active[:40]):
        bz, bx = divmod(int(blk), nbx)
        for lvl in range(max_mip + 1):
            side = 16 >> lvl
            for b in range(L // W):
                # float32 brick rows: the S values of the row's voxels, then their chi values
                rows = bricks[b, r, off[lvl]:off[lvl] + side * side].reshape(side, 2, side, W)
                rec = np.concatenate([rows[:, 0].reshape(-1, W), rows[:, 1].reshape(-1, W)], axis=1)  # [side*side][2W]
                e_m = levels[lvl][0][b * W:(b + 1) * W, bz * side:(bz + 1) * side, bx * side:(bx + 1) * side]
                c_m = levels[lvl][1][b * W:(b + 1) * W, bz * side:(bz + 1) * side, bx * side:(bx + 1) * side]
                c_ref = c_m.reshape(W, -1).T
                s_ref = np.where(c_ref > 0, e_m.reshape(W, -1).T / np.where(c_ref > 0, c_ref, 1), e_m.reshape(W, -1).T)
                assert_rel(rec[:, W:], c_ref, 2e-6, f"chi level {lvl}")
                assert_rel(rec[:, :W], s_ref, 2e-6, f"S level {lvl}")


@pytest.mark.parametrize("max_mip,te", [(0, 1.0), (3, 1e-2), (3, 1.0), (2, 1e-3)])
def test_hdda_matches_expanded_oracle(ctx, max_mip, te):
    nx, nz, L, W = 128, 96, 16, 8
    m = line_model(nx, nz, L, synth.SEED_BASE + 420)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    dirs, w = synth.directions(16)
    grid, mp, J, I, seg = gpu_pipeline(ctx, nx, nz, eg, cg, W, max_mip, te, te, dirs=dirs, w=w)
    o = oracle_pipeline(er, cr, W, max_mip, te, te, dirs=dirs, w=w)
    if max_mip > 0:
        robust = robust_level_mask(o["stats"], o["lev"], W, 16, max_mip, te, te, 0.25)
        assert robust.all(), "this input has a block whose level is within rounding of a threshold"
    p = o["probes"]
    assert_rel(I.cpu().numpy()[:, :, p], o["I"], what=f"I max_mip={max_mip}")
    assert_rel(J.cpu().numpy()[:, p], o["J"], what=f"J max_mip={max_mip}")
    # cells of empty blocks are not probes and stay zero
    mask = np.ones(nx * nz, bool)
    mask[p] = False
    assert not J.cpu().numpy()[:, mask].any()


@pytest.mark.parametrize("W,L", [(1, 3), (2, 6), (4, 12)])
def test_hdda_narrow_batches_match_expanded_oracle(ctx, W, L):
    """Float32 brick rows at batch widths 1, 2 and 4 (scalar, 64-bit and 128-bit
    record loads, ragged last batch): the accelerated solve against the float64
    oracle on the expanded grid, at levels 0-3 with the paper's IoD threshold."""
    nx, nz, max_mip, te = 96, 64, 3, 1.0
    m = line_model(nx, nz, L, synth.SEED_BASE + 425)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    dirs, w = synth.directions(12)
    grid, mp, J, I, seg = gpu_pipeline(ctx, nx, nz, eg, cg, W, max_mip, te, te, dirs=dirs, w=w)
    o = oracle_pipeline(er, cr, W, max_mip, te, te, dirs=dirs, w=w)
    robust = robust_level_mask(o["stats"], o["lev"], W, 16, max_mip, te, te, 0.25)
    assert robust.all(), "this input has a block whose level is within rounding of a threshold"
    assert (o["lev"] > 0).any(), "the test wants coarse levels"
    p = o["probes"]
    assert_rel(I.cpu().numpy()[:, :, p], o["I"], what=f"I W={W}")
    assert_rel(J.cpu().numpy()[:, p], o["J"], what=f"J W={W}")


def test_hdda_level0_equals_plain_dense(ctx):
    """Sparse skipping alone (max_mip 0) reproduces the plain full-resolution solve
    at every probe: empty blocks hold eta = chi = 0."""
    from paper_2511_08498_gb300 import api
    nx, nz, L = 96, 64, 8
    m = line_model(nx, nz, L, synth.SEED_BASE + 430)
    eg, cg = gpu_line_eta_chi(ctx, m)
    dirs, w = synth.directions(12)
    grid, mp, Js, _, seg_s = gpu_pipeline(ctx, nx, nz, eg, cg, 8, 0, 1.0, 1.0, dirs=dirs, w=w, want_I=False)
    planes = api.pack_planes(ctx, eg, cg, 8)
    Jd, _, seg_d = api.formal_solve_dense(ctx, nx, nz, L, 8, planes, dirs, w, count_segments=True)
    ctx.check()
    er, cr = oracle_line_eta_chi(m)
    p = omips.probes_of_blocks(omips.block_empty(er, cr, 16), 16)
    assert_rel(Js.cpu().numpy()[:, p], Jd.cpu().numpy()[:, p].astype(np.float64), 2e-6, "sparse vs dense")
    assert int(seg_s.item()) < int(seg_d.item())


def test_fig5_block_map(ctx):
    """The adapted grid of the paper's HDDA figure, scaled to 16^2 blocks: a 4 x 4
    block grid with blocks 0, 1, 2, 4, 8, 12, 15 empty, block 9 one level coarser
    than its neighbours' full resolution... expressed here as levels 0 / 1 / 2."""
    n = 64
    med = synth.random_medium(n, n, 8, seed=synth.SEED_BASE + 440, zero_frac=0.0, emitter_frac=0.0)
    eta, chi = med["eta"].copy(), med["chi"].copy()
    empty_blocks = [0, 1, 2, 4, 8, 12, 15]
    for k in empty_blocks:
        bz, bx = divmod(k, 4)
        eta[:, bz * 16:(bz + 1) * 16, bx * 16:(bx + 1) * 16] = 0
        chi[:, bz * 16:(bz + 1) * 16, bx * 16:(bx + 1) * 16] = 0
    cap = np.zeros((4, 4), np.int8)
    cap[2, 1] = 1   # block 9
    cap[2, 2] = 2   # block 10
    dirs, w = synth.directions(16)
    eg = torch.from_numpy(eta.reshape(8, -1)).cuda()
    cg = torch.from_numpy(chi.reshape(8, -1)).cuda()
    inf = float("inf")
    grid, mp, J, I, _ = gpu_pipeline(ctx, n, n, eg, cg, 8, 2, inf, inf, cm=inf, level_cap=cap, dirs=dirs, w=w)
    o = oracle_pipeline(eta, chi, 8, 2, inf, inf, cm=inf, level_cap=cap, dirs=dirs, w=w)
    assert o["lev"][0].tolist() == [[-1, -1, -1, 0], [-1, 0, 0, 0], [-1, 1, 2, 0], [-1, 0, 0, -1]]
    from paper_2511_08498_gb300 import api
    assert api.unpack_states(mp.words.cpu().numpy(), 16).reshape(4, 4).tolist() == o["lev"][0].tolist()
    p = o["probes"]
    assert_rel(I.cpu().numpy()[:, :, p], o["I"], what="I fig5")


def test_homogeneous_medium_reaches_top_level_and_matches_plain(ctx):
    """Section 1.1: with homogeneous parameters the averaged solution is the true one."""
    n = 64
    eta = np.full((8, n, n), 0.35, np.float32)
    chi = np.full((8, n, n), 0.2, np.float32)
    dirs, w = synth.directions(8)
    eg = torch.from_numpy(eta.reshape(8, -1)).cuda()
    cg = torch.from_numpy(chi.reshape(8, -1)).cuda()
    grid, mp, J, I, seg = gpu_pipeline(ctx, n, n, eg, cg, 8, 4, 1e-6, 1e-6, dirs=dirs, w=w)
    from paper_2511_08498_gb300 import api
    assert (api.unpack_states(mp.words.cpu().numpy(), 16) == 4).all()
    Jr = lc.formal_solve(eta, chi, dirs, w)
    assert_rel(J.cpu().numpy(), Jr, what="homogeneous")


def test_all_empty_and_single_block_grids(ctx):
    from paper_2511_08498_gb300 import api
    dirs, w = synth.directions(8)
    z = torch.zeros((2, 32 * 32), device="cuda")
    grid, mp, J, _, seg = gpu_pipeline(ctx, 32, 32, z, z, 2, 3, 1.0, 1.0, dirs=dirs, w=w, want_I=False)
    assert grid.n_active() == 0 and not J.any() and int(seg.item()) == 0
    med = synth.random_medium(16, 16, 3, seed=synth.SEED_BASE + 450)
    eg = torch.from_numpy(med["eta"].reshape(3, -1)).cuda()
    cg = torch.from_numpy(med["chi"].reshape(3, -1)).cuda()
    grid, mp, J, I, _ = gpu_pipeline(ctx, 16, 16, eg, cg, 4, 4, 0.5, 0.5, dirs=dirs, w=w)
    o = oracle_pipeline(med["eta"], med["chi"], 4, 4, 0.5, 0.5, dirs=dirs, w=w)
    assert grid.n_active() == 1
    assert_rel(J.cpu().numpy(), o["J"], what="single block")


def test_axis_parallel_rays_through_levels(ctx):
    nx, nz, L = 96, 80, 8
    m = line_model(nx, nz, L, synth.SEED_BASE + 460)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    dirs, w = synth.directions(8, offset=0.0)
    grid, mp, J, I, _ = gpu_pipeline(ctx, nx, nz, eg, cg, 8, 3, 1.0, 1.0, dirs=dirs, w=w)
    o = oracle_pipeline(er, cr, 8, 3, 1.0, 1.0, dirs=dirs, w=w)
    robust = robust_level_mask(o["stats"], o["lev"], 8, 16, 3, 1.0, 1.0, 0.25)
    assert robust.all()
    assert_rel(I.cpu().numpy()[:, :, o["probes"]], o["I"], what="axis-parallel")


@pytest.mark.parametrize("band", [[5.3, 21.7, 60.1], [0.0], [], [2.2, 2.2, 9.9]])
def test_distance_limited_levels_match_oracle(ctx, band):
    """Section 4.1's near-field-at-full-resolution limit, long-characteristics form:
    a block first entered at ray parameter t uses at most the number of thresholds <= t."""
    from paper_2511_08498_gb300 import api
    nx, nz, L, W = 128, 96, 16, 8
    m = line_model(nx, nz, L, synth.SEED_BASE + 470)
    eg, cg = gpu_line_eta_chi(ctx, m)
    er, cr = oracle_line_eta_chi(m)
    dirs, w = synth.directions(16)
    te = 1.0
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, 3, te, te, 0.25, log_mean=False)
    J, I, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w, want_intensity=True, band=band)
    ctx.check()
    levels, passes, st = omips.mip_chain(er, cr, 3, te, te, 0.25, mean="linear", stats=True)
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W)
    assert robust_level_mask(st, lev, W, 16, 3, te, te, 0.25).all()
    probes = omips.probes_of_blocks(empty, 16)
    Jr, Ir = lc.formal_solve_banded(levels, lev, 16, W, band, dirs, w, probes, want_intensity=True)
    assert_rel(I.cpu().numpy()[:, :, probes], Ir, what=f"I band={band}")
    assert_rel(J.cpu().numpy()[:, probes], Jr, what=f"J band={band}")
