"""Edge cases of the 3D and radiance-cascade entry points against the oracles.

* argument checks: sizes that are not whole blocks or not divisible by the top
  cascade's spacing, levels above the 3D or chain maximum, too many cascades,
  a level cap above the bricks' top level -- each rejected before any launch;
* a 3D grid of a single 8^3 block with axis-parallel and corner rays;
* a 3D grid whose blocks are all empty: J is zero everywhere;
* one cascade with one direction and an interval past the grid: the cascade
  solve is the long-characteristics solve of that direction;
* a 2D grid with a single non-empty block in the cascade solve.
"""

import numpy as np
import pytest

import synth
from oracle import lc, lc3, mips as omips, mips3, rc

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(a.shape[0], -1)).cuda()


def test_argument_checks(ctx):
    from paper_2511_08498_gb300 import api
    from paper_2511_08498_gb300._native import DexError
    e = torch.ones((1, 12 * 8 * 8), device="cuda")
    with pytest.raises(DexError):
        api.grid3_build(ctx, 12, 8, 8, e, e)                     # 12 is not a whole number of blocks
    e = torch.ones((1, 8 * 8 * 8), device="cuda")
    g = api.grid3_build(ctx, 8, 8, 8, e, e)
    with pytest.raises(DexError):
        api.mips3_build(ctx, g, e, e, 8, 4, 1.0, 1.0)             # level 4 does not exist in 3D
    e2 = torch.ones((1, 48 * 48), device="cuda")
    g2 = api.grid_build(ctx, 48, 48, e2, e2)
    mp = api.mips_build(ctx, g2, e2, e2, 8, 2, 1.0, 1.0)
    with pytest.raises(DexError):
        api.rc_solve(ctx, g2, mp, n_cascades=6)                   # 48 is not a multiple of 32
    with pytest.raises(DexError):
        api.rc_solve(ctx, g2, mp, n_cascades=9)
    with pytest.raises(DexError):
        api.rc_solve(ctx, g2, mp, n_cascades=3, level_cap=[0, 1, 3])  # above the chains' level 2
    ctx.check()


def test_3d_single_block(ctx):
    from paper_2511_08498_gb300 import api
    L = 8
    m = synth.random_medium3(8, 8, 8, L, seed=synth.SEED_BASE + 500)
    eg, cg = dev(m["eta"]), dev(m["chi"])
    d = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1], [-1, 1, -1]]
    dirs = (np.array(d, np.float64) / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    w = np.full(len(d), 1.0 / len(d), np.float32)
    grid = api.grid3_build(ctx, 8, 8, 8, eg, cg)
    mp = api.mips3_build(ctx, grid, eg, cg, 8, 3, 1e30, 1e30, 0.25)
    J, _, _ = api.formal_solve_hdda3(ctx, grid, mp, dirs, w, i_bc=0.2)
    ctx.check()
    e, c = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    levels, passes = mips3.mip_chain(e, c, 3, 1e30, 1e30, 0.25, mean="linear")
    lev = mips3.block_levels(passes, mips3.block_empty(e, c, 8), 8, 8)
    Jr = lc3.formal_solve(*mips3.expand(levels, lev, 8), dirs, w, i_bc=0.2)
    assert rel(J.cpu().numpy(), Jr).max() < 1e-5


def test_3d_all_blocks_empty(ctx):
    from paper_2511_08498_gb300 import api
    z = torch.zeros((2, 16 * 16 * 8), device="cuda")
    grid = api.grid3_build(ctx, 16, 16, 8, z, z)
    assert grid.n_active() == 0
    mp = api.mips3_build(ctx, grid, z, z, 2, 3, 1.0, 1.0, 0.25)
    dirs, w = synth.directions3(4, 2)
    J, _, _ = api.formal_solve_hdda3(ctx, grid, mp, dirs, w, i_bc=1.0)
    ctx.check()
    assert (J == 0).all()


def test_one_cascade_one_direction_is_long_characteristics(ctx):
    from paper_2511_08498_gb300 import api
    nx, nz, L = 48, 32, 4
    m = synth.random_medium(nx, nz, L, seed=synth.SEED_BASE + 510)
    eg, cg = dev(m["eta"]), dev(m["chi"])
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, 4, 0, 1e30, 1e30, 0.25)
    dirs = synth.rc_directions(1, 1)
    J, _ = api.rc_solve(ctx, grid, mp, n_cascades=1, n0=1, t0=1e4, level_cap=[0], dirs=dirs, i_bc=0.3)
    ctx.check()
    e, c = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    probes = omips.probes_of_blocks(omips.block_empty(e, c, 16), 16)
    Jr = lc.formal_solve(e, c, dirs[0], [1.0], probes=probes, i_bc=0.3)
    assert rel(J.cpu().numpy()[:, probes], Jr).max() < 1e-5


def test_cascades_with_a_single_non_empty_block(ctx):
    from paper_2511_08498_gb300 import api
    nx = nz = 64
    L = 8
    rng = np.random.default_rng(7)
    chi = np.zeros((L, nz, nx), np.float32)
    chi[:, 16:32, 32:48] = rng.uniform(0.05, 2.0, (L, 16, 16))
    eta = (chi * rng.uniform(0.5, 2.0, (L, nz, nx))).astype(np.float32)
    eg, cg = dev(eta), dev(chi)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    assert grid.n_active() == 1
    mp = api.mips_build(ctx, grid, eg, cg, 8, 2, 1e30, 1e30, 0.25)
    caps = [0, 1, 2, 2]
    J, _ = api.rc_solve(ctx, grid, mp, n_cascades=4, n0=4, level_cap=caps, dirs=synth.rc_directions(4, 4),
                        i_bc=0.5)
    ctx.check()
    e, c = eta.astype(np.float64), chi.astype(np.float64)
    empty = omips.block_empty(e, c, 16)
    levels, passes = omips.mip_chain(e, c, 2, 1e30, 1e30, 0.25, mean="linear")
    lev = omips.block_levels(passes, empty, 16, 8)
    grids = [omips.expand(levels, np.where(lev >= 0, np.minimum(lev, caps[i]), -1), 8) for i in range(4)]
    Jr = rc.rc_solve(grids, 4, 4, synth.rc_directions(4, 4), i_bc=0.5)
    probes = omips.probes_of_blocks(empty, 16)
    assert rel(J.cpu().numpy()[:, probes], Jr[:, probes]).max() < 1e-5
    outside = np.setdiff1d(np.arange(nx * nz), probes)
    assert (J.cpu().numpy()[:, outside] == 0).all()
