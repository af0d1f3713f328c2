"""One walk per ray for two wavelength batches b and n_batch - 1 - b
(DEX_TRAVERSAL_SHARED) vs the float64 oracle and vs one walk per batch.

Each batch keeps its own block levels (Section 4.1): in a block the shared walk
steps at the finer of the two batches' levels and a coarser batch integrates
its voxel once, when the walk leaves it, over the length between the same two
planes its own walk would use.  So:

* against the oracle (plain solve on the grid expanded with each batch's
  levels, or the distance-banded solve): 1e-5 relative, the accelerated bar;
* against the per-batch walk on the same bricks: the same plane parameters and
  the same updates in the same order -- J and I within 2e-6 relative (bit-equal
  in practice) and the same executed segment count;
* the inputs are checked to give the batches different level maps (otherwise
  the lazy integration of coarse batches would not be exercised), and to have
  no block level within rounding of a threshold.
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
    c.set_traversal(False)


def model(L, seed, shift):
    m = synth.sparse_line_atmosphere(NX, NZ, n_lambda=L, seed=synth.SEED_BASE + seed)
    # line centre moved off the middle of the wavelength grid: mirrored batches then
    # see different parts of the line and take different levels
    m["dlam"] = (m["dlam"] + shift).astype(m["dlam"].dtype)
    er, cr = lines.line_eta_chi(m["chi_c"], m["s_c"], m["s_l"], m["ratio"], m["dld"], m["dlam"])
    return m, er, cr


def gpu_solve(ctx, m, L, thr, band, storage, shared, dirs, w):
    from paper_2511_08498_gb300 import api
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    grid = api.grid_build(ctx, NX, NZ, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, 3, thr, thr, 0.25, log_mean=False, storage=storage)
    ctx.set_traversal(shared)
    J, I, seg = api.formal_solve_hdda(ctx, grid, mp, dirs, w, want_intensity=True, count_segments=True, band=band)
    ctx.check()
    ctx.set_traversal(False)
    glev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks).reshape(-1, NZ // 16, NX // 16)
    return J.cpu().numpy(), I.cpu().numpy(), int(seg.item()), glev


# (wavelengths, seed, IoD threshold, distance limits, line-centre shift in grid
# units): 5 batches (pairs 0-4, 1-3 and batch 2 alone), 4.5 batches (a ragged
# last batch), 3 batches, 4 batches
CASES = [(40, 480, 1e-2, None, 5.0), (36, 481, 1.0, [5.3, 21.7, 60.1], 0.0), (24, 482, 1e-2, [2.2, 9.9], -3.5),
         (32, 483, 1e30, [6.0, 24.0, 96.0], 2.0)]


@pytest.mark.parametrize("L,seed,thr,band,shift", CASES)
def test_shared_walk_matches_oracle(ctx, L, seed, thr, band, shift):
    m, er, cr = model(L, seed, shift)
    dirs, w = synth.directions(12)
    J, I, seg, glev = gpu_solve(ctx, m, L, thr, band, 0, True, dirs, w)
    levels, passes, st = omips.mip_chain(er, cr, 3, thr, thr, 0.25, mean="linear", stats=True)
    empty = omips.block_empty(er, cr, 16)
    lev = omips.block_levels(passes, empty, 16, W)
    assert robust_level_mask(st, lev, W, 16, 3, thr, thr, 0.25).all()
    np.testing.assert_array_equal(glev, lev)
    act, nb = lev[0] >= 0, lev.shape[0]
    assert any(not np.array_equal(lev[b][act], lev[nb - 1 - b][act]) for b in range(nb // 2)), \
        "the batches sharing a walk have equal level maps: the per-batch integration is not exercised"
    probes = omips.probes_of_blocks(empty, 16)
    if band is None:
        e2, c2 = omips.expand(levels, lev, W)
        Jr, Ir = lc.formal_solve(e2, c2, dirs, w, probes=probes, want_intensity=True)
    else:
        Jr, Ir = lc.formal_solve_banded(levels, lev, 16, W, band, dirs, w, probes, want_intensity=True)
    assert rel(I[:, :, probes], Ir).max() < 1e-5
    assert rel(J[:, probes], Jr).max() < 1e-5
    zero = Jr == 0
    assert np.array_equal(J[:, probes][zero], Jr[zero])


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("L,seed,thr,band,shift", CASES[:2])
def test_shared_walk_equals_per_batch_walk(ctx, storage, L, seed, thr, band, shift):
    m, _, _ = model(L, seed, shift)
    dirs, w = synth.directions(12, offset=0.0)   # axis-parallel and diagonal rays included
    Js, Is, ss, _ = gpu_solve(ctx, m, L, thr, band, storage, True, dirs, w)
    Jp, Ip, sp, _ = gpu_solve(ctx, m, L, thr, band, storage, False, dirs, w)
    assert rel(Is, Ip).max() < 2e-6
    assert rel(Js, Jp).max() < 2e-6
    assert ss == sp


def test_traversal_mode_is_checked(ctx):
    from paper_2511_08498_gb300 import _native, api
    assert _native.lib().dex_ctx_set_traversal(ctx.handle, 3) == 1   # DEX_ERR_ARG
    ctx.set_traversal(False)
