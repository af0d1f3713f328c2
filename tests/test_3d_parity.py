"""3D path (8^3 blocks, levels 0..3) on the GPU vs the float64 3D oracle.

* plain solve, every cell and a probe list, ragged sizes, W = 1, 4, 8: I and J
  within 1e-5 relative; the segment count equals the oracle's exactly;
* axis-parallel rays and rays through cube corners (every tie of the DDA);
* sparsity map and Morton layout: bit-exact;
* block levels with unlimited averaging: exact; at IoD 0.1 exact wherever the
  oracle's decision is not within 1e-4 of a threshold;
* accelerated solve against the oracle on its own MIP chains (expanded, and
  distance-banded): 1e-5 relative;
* at level 0 the accelerated solve reproduces the plain solve bit for bit
  (empty blocks add exact zeros, and both walk the same planes);
* bfloat16 bricks at level 0 against the oracle on bfloat16-rounded records.
"""

import numpy as np
import pytest

import synth
from levels_util import robust_level_mask3
from oracle import lc3, lines, mips3

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def assert_rel(gpu, ref, rtol=1e-5, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    zero = ref == 0
    assert np.array_equal(gpu[zero], ref[zero]), f"{what}: exact zeros differ"
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-30)
    worst = np.unravel_index(np.argmax(rel), rel.shape)
    assert rel.max() <= rtol, f"{what}: max rel err {rel.max():.3e} at {worst}: gpu {gpu[worst]} ref {ref[worst]}"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(a.shape[0], -1)).cuda()


def axis_and_corner_dirs():
    d = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    d += [[sx, sy, sz] for sx in (1, -1) for sy in (1, -1) for sz in (1, -1)]
    d = np.array(d, dtype=np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32), np.full(len(d), 1.0 / len(d), np.float32)


@pytest.mark.parametrize("W", [1, 4, 8])
def test_dense3_every_cell_ragged(ctx, W):
    from paper_2511_08498_gb300 import api
    nx, ny, nz, L = 23, 19, 13, 5
    m = synth.random_medium3(nx, ny, nz, L, seed=synth.SEED_BASE + 140 + W)
    dirs, w = synth.directions3(8, 4)
    planes = api.pack_planes(ctx, dev(m["eta"]), dev(m["chi"]), W)
    J, I, seg = api.formal_solve_dense3(ctx, nx, ny, nz, L, W, planes, dirs, w, i_bc=0.3, want_intensity=True,
                                        count_segments=True)
    ctx.check()
    Jr, Ir = lc3.formal_solve(m["eta"], m["chi"], dirs, w, i_bc=0.3, want_intensity=True)
    assert_rel(I.cpu().numpy(), Ir, what="I")
    assert_rel(J.cpu().numpy(), Jr, what="J")
    n_batch = -(-L // W)
    full = lc3.count_segments((nx, ny, nz), dirs, np.arange(nx * ny * nz, dtype=np.int32))
    assert int(seg.item()) == n_batch * full


def test_dense3_probe_list_and_degenerate_rays(ctx):
    from paper_2511_08498_gb300 import api
    nx, ny, nz, L = 16, 12, 10, 8
    m = synth.random_medium3(nx, ny, nz, L, seed=synth.SEED_BASE + 150)
    dirs, w = axis_and_corner_dirs()
    d2, w2 = synth.directions3(4, 3, offset=0.0)   # mu = 0 nodes: rays in the x-z plane, axis-parallel ones
    dirs = np.concatenate([dirs, d2])
    w = np.concatenate([w, w2]) * 0.5
    probes = np.sort(np.random.default_rng(2).choice(nx * ny * nz, 300, replace=False)).astype(np.int32)
    planes = api.pack_planes(ctx, dev(m["eta"]), dev(m["chi"]), 8)
    J, I, _ = api.formal_solve_dense3(ctx, nx, ny, nz, L, 8, planes, dirs, w, probes=torch.from_numpy(probes).cuda(),
                                      i_bc=0.0, want_intensity=True)
    ctx.check()
    Jr, Ir = lc3.formal_solve(m["eta"], m["chi"], dirs, w, probes=probes, want_intensity=True)
    assert_rel(I.cpu().numpy(), Ir, what="I")
    assert_rel(J.cpu().numpy(), Jr, what="J")


def line3(ctx, nx, ny, nz, L, seed, empty_frac=0.4):
    from paper_2511_08498_gb300 import api
    m = synth.sparse_line_atmosphere3(nx, ny, nz, n_lambda=L, seed=seed, empty_frac=empty_frac)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    er, cr = lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])
    # the oracle takes the GPU's float32 MIP-0 values (line synthesis is pinned separately)
    e32 = eg.cpu().numpy().reshape(er.shape).astype(np.float64)
    c32 = cg.cpu().numpy().reshape(cr.shape).astype(np.float64)
    assert np.allclose(e32, er, rtol=2e-6, atol=0) and np.allclose(c32, cr, rtol=2e-6, atol=0)
    return eg, cg, e32, c32


def test_grid3_layout_bit_exact(ctx):
    from paper_2511_08498_gb300 import api
    nx, ny, nz = 64, 48, 40
    eg, cg, er, cr = line3(ctx, nx, ny, nz, 6, synth.SEED_BASE + 160)
    grid = api.grid3_build(ctx, nx, ny, nz, eg, cg)
    ctx.check()
    empty = mips3.block_empty(er, cr, 8)
    active, offset = mips3.block_layout(empty)
    n = grid.n_active()
    assert 0 < n < grid.n_blocks and n == active.size
    assert np.array_equal(grid.active.cpu().numpy()[:n], active)
    assert np.array_equal(grid.block_offset.cpu().numpy(), offset.reshape(-1))


def _sparse(ctx, nx, ny, nz, eg, cg, W, max_mip, iod, dirs, w, band=None, log_mean=False, storage=0, want_I=True):
    from paper_2511_08498_gb300 import api
    grid = api.grid3_build(ctx, nx, ny, nz, eg, cg)
    mp = api.mips3_build(ctx, grid, eg, cg, W, max_mip, iod, iod, 0.25, log_mean=log_mean, storage=storage)
    J, I, seg = api.formal_solve_hdda3(ctx, grid, mp, dirs, w, band=band, want_intensity=want_I,
                                       count_segments=True)
    ctx.check()
    lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks).reshape(-1, nz // 8, ny // 8, nx // 8)
    return grid, lev, J.cpu().numpy(), None if I is None else I.cpu().numpy(), int(seg.item())


@pytest.mark.parametrize("W,log_mean", [(8, False), (4, True), (1, False)])
def test_hdda3_unlimited_levels_against_expanded_oracle(ctx, W, log_mean):
    nx, ny, nz, L = 48, 40, 32, 8
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 170 + W)
    dirs, w = synth.directions3(8, 4)
    _, lev, J, I, _ = _sparse(ctx, nx, ny, nz, eg, cg, W, 3, 1e30, dirs, w, log_mean=log_mean)
    levels, passes = mips3.mip_chain(er, cr, 3, 1e30, 1e30, 0.25, mean="log" if log_mean else "linear")
    empty = mips3.block_empty(er, cr, 8)
    lev_r = mips3.block_levels(passes, empty, 8, W)
    assert np.array_equal(lev, lev_r)
    # unlimited averaging: every block reaches level 3 except some at the transition
    # surface, whose groups mix empty and filled cells (they pass only where thin)
    assert (lev_r[lev_r >= 0] == 3).mean() > 0.5
    probes = mips3.probes_of_blocks(empty, 8)
    Jr, Ir = lc3.formal_solve(*mips3.expand(levels, lev_r, W), dirs, w, probes=probes, want_intensity=True)
    assert_rel(I[:, :, probes], Ir, what="I")
    assert_rel(J[:, probes], Jr, what="J")


def test_hdda3_distance_banded_against_oracle(ctx):
    nx, ny, nz, L = 56, 48, 40, 13                 # ragged last wavelength batch (13 = 8 + 5)
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 180)
    dirs, w = synth.directions3(8, 4)
    band = [3.0, 9.0, 20.0]
    _, lev, J, I, _ = _sparse(ctx, nx, ny, nz, eg, cg, 8, 3, 1e30, dirs, w, band=band)
    levels, passes = mips3.mip_chain(er, cr, 3, 1e30, 1e30, 0.25, mean="linear")
    empty = mips3.block_empty(er, cr, 8)
    lev_r = mips3.block_levels(passes, empty, 8, 8)
    assert np.array_equal(lev, lev_r)
    probes = mips3.probes_of_blocks(empty, 8)
    Jr, Ir = lc3.formal_solve_banded(levels, lev_r, 8, 8, band, dirs, w, probes, want_intensity=True)
    assert_rel(I[:, :, probes], Ir, what="I")
    assert_rel(J[:, probes], Jr, what="J")


def test_hdda3_threshold_levels(ctx):
    nx, ny, nz, L = 64, 48, 40, 8
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 190)
    dirs, w = synth.directions3(4, 2)
    _, lev, J, _, _ = _sparse(ctx, nx, ny, nz, eg, cg, 8, 3, 0.1, dirs, w, band=[4.0, 12.0, 24.0], want_I=False)
    levels, passes, st = mips3.mip_chain(er, cr, 3, 0.1, 0.1, 0.25, mean="linear", stats=True)
    empty = mips3.block_empty(er, cr, 8)
    lev_r = mips3.block_levels(passes, empty, 8, 8)
    robust = robust_level_mask3(st, lev_r, 8, 3, 0.1, 0.1, 0.25)
    assert robust.mean() > 0.95
    assert np.array_equal(lev[robust], lev_r[robust])
    assert len(np.unique(lev_r[lev_r >= 0])) == 4     # the threshold selects every level somewhere
    if np.array_equal(lev, lev_r):
        probes = mips3.probes_of_blocks(empty, 8)
        Jr = lc3.formal_solve_banded(levels, lev_r, 8, 8, [4.0, 12.0, 24.0], dirs, w, probes)
        assert_rel(J[:, probes], Jr, what="J")


def test_hdda3_level0_is_the_plain_solve_bit_for_bit(ctx):
    from paper_2511_08498_gb300 import api
    nx, ny, nz, L = 48, 40, 32, 8
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 200)
    dirs, w = synth.directions3(8, 4)
    d2, w2 = axis_and_corner_dirs()
    dirs, w = np.concatenate([dirs, d2]), np.concatenate([w, w2])
    _, _, J, I, seg = _sparse(ctx, nx, ny, nz, eg, cg, 8, 0, 1e30, dirs, w)
    empty = mips3.block_empty(er, cr, 8)
    probes = mips3.probes_of_blocks(empty, 8)
    planes = api.pack_planes(ctx, eg, cg, 8)
    Jd, Id, _ = api.formal_solve_dense3(ctx, nx, ny, nz, L, 8, planes, dirs, w,
                                        probes=torch.from_numpy(probes).cuda(), want_intensity=True)
    ctx.check()
    assert np.array_equal(J[:, probes], Jd.cpu().numpy())
    assert np.array_equal(I[:, :, probes], Id.cpu().numpy())


def _bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def test_hdda3_bf16_bricks_level0(ctx):
    nx, ny, nz, L = 40, 32, 32, 8
    eg, cg, er, cr = line3(ctx, nx, ny, nz, L, synth.SEED_BASE + 210)
    dirs, w = synth.directions3(4, 4)
    _, _, J, _, _ = _sparse(ctx, nx, ny, nz, eg, cg, 8, 0, 1e30, dirs, w, storage=1, want_I=False)
    e32, c32 = er.astype(np.float32), cr.astype(np.float32)
    S = np.where(c32 > 0, e32 / np.where(c32 > 0, c32, 1), 0).astype(np.float32)
    Sb, cb = _bf16_round(S).astype(np.float64), _bf16_round(c32).astype(np.float64)
    empty = mips3.block_empty(er, cr, 8)
    probes = mips3.probes_of_blocks(empty, 8)
    Jr = lc3.formal_solve(Sb * cb, cb, dirs, w, probes=probes)
    assert_rel(J[:, probes], Jr, what="J")
