"""Edge cases of the solvers at the limits of their arguments, against the oracle.

* the largest quadrature (256 directions) in both solvers; 257 is rejected;
* a ragged last wavelength batch (13 wavelengths in batches of 8) through the
  accelerated path;
* grids of a single block, of a single block row or column, and of two
  blocks, with axis-parallel and diagonal rays at the coarsest level (4);
* one wavelength with W = 8 (seven padding lanes).
"""

import numpy as np
import pytest

import synth
from oracle import lc, lines, mips as omips

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-30)


def line_case(ctx, nx, nz, L, seed):
    from paper_2511_08498_gb300 import api
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=seed)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    er, cr = lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])
    return eg, cg, er, cr


def accelerated(ctx, nx, nz, eg, cg, W, max_mip, iod, dirs, w, band):
    from paper_2511_08498_gb300 import api
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mips = api.mips_build(ctx, grid, eg, cg, W, max_mip, iod, iod, 0.25, log_mean=False)
    J, I, _ = api.formal_solve_hdda(ctx, grid, mips, dirs, w, band=band, want_intensity=True)
    ctx.check()
    return J.cpu().numpy(), I.cpu().numpy()


def oracle_accelerated(er, cr, W, max_mip, iod, dirs, w, band):
    levels, passes = omips.mip_chain(er, cr, max_mip, iod, iod, 0.25, mean="linear")
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W, n_lambda=er.shape[0])
    probes = omips.probes_of_blocks(empty, 16)
    if band is None:  # no distance limit: every block at its level everywhere
        J, I = lc.formal_solve(*omips.expand(levels, lev, W), dirs, w, probes=probes, want_intensity=True)
    else:
        J, I = lc.formal_solve_banded(levels, lev, 16, W, band, dirs, w, probes, want_intensity=True)
    return probes, J, I


def test_largest_quadrature(ctx):
    from paper_2511_08498_gb300 import api
    from paper_2511_08498_gb300._native import DexError
    nx, nz, L = 48, 32, 8
    eg, cg, er, cr = line_case(ctx, nx, nz, L, synth.SEED_BASE + 700)
    dirs, w = synth.directions(256)
    planes = api.pack_planes(ctx, eg, cg, 8)
    J, _, _ = api.formal_solve_dense(ctx, nx, nz, L, 8, planes, dirs, w)
    ctx.check()
    Jr = lc.formal_solve(er, cr, dirs, w)
    assert rel(J.cpu().numpy(), Jr).max() < 1e-5
    Ja, _ = accelerated(ctx, nx, nz, eg, cg, 8, 0, 1.0, dirs, w, None)
    probes = omips.probes_of_blocks(omips.block_empty(er, cr, 16), 16)
    assert rel(Ja[:, probes], Jr[:, probes]).max() < 1e-5
    d257, w257 = synth.directions(257)
    with pytest.raises(DexError):
        api.formal_solve_dense(ctx, nx, nz, L, 8, planes, d257, w257)
    ctx.check()


def test_ragged_wavelength_batch_accelerated(ctx):
    nx, nz, L = 96, 80, 13
    eg, cg, er, cr = line_case(ctx, nx, nz, L, synth.SEED_BASE + 710)
    dirs, w = synth.directions(16)
    J, I = accelerated(ctx, nx, nz, eg, cg, 8, 3, 1e30, dirs, w, [6.0, 24.0, 96.0])
    probes, Jr, Ir = oracle_accelerated(er, cr, 8, 3, 1e30, dirs, w, [6.0, 24.0, 96.0])
    assert J.shape[0] == L
    assert rel(I[:, :, probes], Ir).max() < 1e-5
    assert rel(J[:, probes], Jr).max() < 1e-5


@pytest.mark.parametrize("nx,nz", [(16, 16), (16, 160), (160, 16), (32, 16)])
def test_single_block_row_and_column_grids(ctx, nx, nz):
    L = 8
    rng = np.random.default_rng(nx * 1000 + nz)
    chi = rng.uniform(0.01, 3.0, (L, nz, nx)).astype(np.float32)
    eta = (chi * rng.uniform(0.5, 2.0, (L, nz, nx))).astype(np.float32)
    e, c = torch.from_numpy(eta.reshape(L, -1)).cuda(), torch.from_numpy(chi.reshape(L, -1)).cuda()
    dirs, w = synth.directions(12, offset=0.0)     # axis-parallel and diagonal rays included
    J, I = accelerated(ctx, nx, nz, e, c, 8, 4, 1e30, dirs, w, None)
    probes, Jr, Ir = oracle_accelerated(eta.astype(np.float64), chi.astype(np.float64), 8, 4, 1e30, dirs, w, None)
    assert rel(I[:, :, probes], Ir).max() < 1e-5
    assert rel(J[:, probes], Jr).max() < 1e-5


def test_one_wavelength_in_a_batch_of_eight(ctx):
    from paper_2511_08498_gb300 import api
    nx, nz, L = 64, 48, 1
    eg, cg, er, cr = line_case(ctx, nx, nz, L, synth.SEED_BASE + 720)
    dirs, w = synth.directions(8)
    planes = api.pack_planes(ctx, eg, cg, 8)
    J, _, _ = api.formal_solve_dense(ctx, nx, nz, L, 8, planes, dirs, w)
    ctx.check()
    assert rel(J.cpu().numpy(), lc.formal_solve(er, cr, dirs, w)).max() < 1e-5
    Ja, _ = accelerated(ctx, nx, nz, eg, cg, 8, 2, 1e30, dirs, w, [6.0, 24.0])
    probes, Jr, _ = oracle_accelerated(er, cr, 8, 2, 1e30, dirs, w, [6.0, 24.0])
    assert rel(Ja[:, probes], Jr).max() < 1e-5


def test_misaligned_records_rejected(ctx):
    """W = 8 float32 and bfloat16 records are read with 256-bit loads: planes and bricks
    must be 32-byte aligned, and a 16-byte-aligned view is refused before any launch."""
    from paper_2511_08498_gb300 import api
    from paper_2511_08498_gb300._native import DexError
    nx, nz, L = 64, 48, 8
    eg, cg, _, _ = line_case(ctx, nx, nz, L, synth.SEED_BASE + 730)
    dirs, w = synth.directions(8)
    n = api.planes_floats(nx * nz, L, 8)
    buf = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
    assert buf.data_ptr() % 32 == 0
    with pytest.raises(DexError, match="aligned"):
        api.pack_planes(ctx, eg, cg, 8, out=buf[4:4 + n].view(-1, nx * nz, 16))
    planes = api.pack_planes(ctx, eg, cg, 8, out=buf[8:8 + n].view(-1, nx * nz, 16))  # 32-byte offset: accepted
    J, _, _ = api.formal_solve_dense(ctx, nx, nz, L, 8, planes, dirs, w)
    with pytest.raises(DexError, match="aligned"):
        api.formal_solve_dense(ctx, nx, nz, L, 8, buf[4:4 + n].view(-1, nx * nz, 16), dirs, w)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mips = api.mips_build(ctx, grid, eg, cg, 8, 3, 1e-2, 1e-2, 0.25, log_mean=False)
    nb = mips.bricks.numel()
    shifted = torch.empty(nb + 4, dtype=torch.float32, device="cuda")
    shifted[4:].copy_(mips.bricks.reshape(-1))
    good = mips.bricks
    mips.bricks = shifted[4:]
    with pytest.raises(DexError, match="aligned"):
        api.formal_solve_hdda(ctx, grid, mips, dirs, w)
    mips.bricks = good
    api.formal_solve_hdda(ctx, grid, mips, dirs, w)
    ctx.check()
    # W = 4 records keep the 16-byte rule
    n4 = api.planes_floats(nx * nz, L, 4)
    p4 = api.pack_planes(ctx, eg, cg, 4, out=buf[4:4 + n4].view(-1, nx * nz, 8))
    J4, _, _ = api.formal_solve_dense(ctx, nx, nz, L, 4, p4, dirs, w)
    ctx.check()
    assert torch.equal(J4, J)


def test_grid_above_the_staged_block_table(ctx):
    """W = 8 grids of more than 8192 blocks read block states from the packed words and
    offsets from global memory instead of one staged word per block: accelerated
    solve of a 65536 x 48 grid (12288 blocks) with empty blocks and distance-limited
    levels against the oracle at sampled probes."""
    from paper_2511_08498_gb300 import api
    nx, nz, L, W = 65536, 48, 2, 8
    rng = np.random.default_rng(synth.SEED_BASE + 740)
    x = np.arange(nx)[None, None, :] + 0.5
    z = np.arange(nz)[None, :, None] + 0.5
    chi = (0.05 * (1.5 + np.sin(2 * np.pi * x / 700.0)) * np.exp(-z / 40.0)
           * np.array([1.0, 3.0])[:, None, None]).astype(np.float32)
    chi = np.broadcast_to(chi, (L, nz, nx)).copy()
    eta = (chi * (1.0 + 0.5 * np.cos(2 * np.pi * x / 333.0))).astype(np.float32)
    nbx = nx // 16
    blk = np.arange(nbx)
    empty_cols = (blk % 7 == 3) | (rng.random(nbx) < 0.1)
    for bz in range(nz // 16):
        cols = empty_cols if bz != 1 else (blk % 11 == 5)
        for bx in np.nonzero(cols)[0]:
            chi[:, bz * 16:(bz + 1) * 16, bx * 16:(bx + 1) * 16] = 0.0
            eta[:, bz * 16:(bz + 1) * 16, bx * 16:(bx + 1) * 16] = 0.0
    eg = torch.from_numpy(eta.reshape(L, -1)).cuda()
    cg = torch.from_numpy(chi.reshape(L, -1)).cuda()
    dirs, w = synth.directions(8)
    band = [6.0, 24.0, 96.0]
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    assert grid.n_blocks > 8192
    mips = api.mips_build(ctx, grid, eg, cg, W, 3, 1e30, 1e30, 0.25, log_mean=False)
    J, _, _ = api.formal_solve_hdda(ctx, grid, mips, dirs, w, band=band)
    ctx.check()
    er, cr = eta.astype(np.float64), chi.astype(np.float64)
    levels, passes = omips.mip_chain(er, cr, 3, 1e30, 1e30, 0.25, mean="linear")
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W, n_lambda=L)
    all_probes = omips.probes_of_blocks(empty, 16)
    probes = np.sort(rng.choice(all_probes, 4096, replace=False)).astype(np.int32)
    Jr = lc.formal_solve_banded(levels, lev, 16, W, band, dirs, w, probes)
    assert rel(J.cpu().numpy()[:, probes], Jr).max() < 1e-5
