"""Radiance cascades on the GPU vs the float64 radiance-cascade oracle.

The oracle runs each cascade on the grid its traversal sees: the block levels
min(selected level, the cascade's cap) expanded onto MIP 0 (empty blocks zero).
J is compared at every cell of every non-empty block: 1e-5 relative.

* full resolution (max MIP 0), the static line model, 4 cascades;
* unlimited averaging with per-cascade caps [0, 0, 1, 2];
* a random medium with transparent emitters and a boundary intensity, W = 1 and 4;
* the paper's configuration (6 cascades, n0 = 4, t0 = 1.5, caps [0, 0, 1, 2, 3, 4]
  within levels 0-3) at 128^2, 512^2 and the benchmark's 1024^2;
* bfloat16 bricks at level 0 against the oracle on bfloat16-rounded records.
"""

import numpy as np
import pytest

import synth
from oracle import lines, mips as omips, rc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def assert_rel(gpu, ref, rtol=1e-5, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-30)
    worst = np.unravel_index(np.argmax(rel), rel.shape)
    assert rel.max() <= rtol, f"{what}: max rel err {rel.max():.3e} at {worst}: gpu {gpu[worst]} ref {ref[worst]}"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


def line2(ctx, nx, nz, L, seed):
    from paper_2511_08498_gb300 import api
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=seed)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eg, cg = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    e = eg.cpu().numpy().reshape(L, nz, nx).astype(np.float64)
    c = cg.cpu().numpy().reshape(L, nz, nx).astype(np.float64)
    return eg, cg, e, c


def gpu_rc(ctx, nx, nz, eg, cg, W, max_mip, iod, C, n0, caps, i_bc=0.0, storage=0, log_mean=False):
    from paper_2511_08498_gb300 import api
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, max_mip, iod, iod, 0.25, log_mean=log_mean, storage=storage)
    J, _ = api.rc_solve(ctx, grid, mp, n_cascades=C, n0=n0, level_cap=caps, dirs=synth.rc_directions(n0, C),
                        i_bc=i_bc)
    ctx.check()
    return J.cpu().numpy()


def oracle_rc(e, c, W, max_mip, iod, C, n0, caps, i_bc=0.0, mean="linear"):
    L = e.shape[0]
    empty = omips.block_empty(e, c, 16)
    if max_mip > 0:
        levels, passes = omips.mip_chain(e, c, max_mip, iod, iod, 0.25, mean=mean)
    else:
        levels, passes = [(e, c)], []
    lev = omips.block_levels(passes, empty, 16, W, n_lambda=L)
    grids = []
    for i in range(C):
        li = np.where(lev >= 0, np.minimum(lev, caps[i]), -1)
        grids.append(omips.expand(levels, li, W))
    J = rc.rc_solve(grids, C, n0, synth.rc_directions(n0, C), i_bc=i_bc)
    return J, omips.probes_of_blocks(empty, 16)


def test_rc_full_resolution(ctx):
    nx, nz, L = 64, 48, 8
    eg, cg, e, c = line2(ctx, nx, nz, L, synth.SEED_BASE + 400)
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 0, 1e30, 4, 4, [0, 0, 0, 0])
    Jr, probes = oracle_rc(e, c, 8, 0, 1e30, 4, 4, [0, 0, 0, 0])
    assert_rel(J[:, probes], Jr[:, probes], what="J")
    empty_cells = np.setdiff1d(np.arange(nx * nz), probes)
    assert (J[:, empty_cells] == 0).all()


def test_rc_mipmapped_with_cascade_caps(ctx):
    nx, nz, L = 96, 64, 13
    eg, cg, e, c = line2(ctx, nx, nz, L, synth.SEED_BASE + 410)
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 3, 1e30, 4, 4, [0, 0, 1, 2])
    Jr, probes = oracle_rc(e, c, 8, 3, 1e30, 4, 4, [0, 0, 1, 2])
    assert_rel(J[:, probes], Jr[:, probes], what="J")


@pytest.mark.parametrize("W", [1, 4])
def test_rc_random_medium_with_boundary(ctx, W):
    nx, nz, L = 48, 32, 5
    m = synth.random_medium(nx, nz, L, seed=synth.SEED_BASE + 420 + W)
    eg = torch.from_numpy(m["eta"].reshape(L, -1)).cuda()
    cg = torch.from_numpy(m["chi"].reshape(L, -1)).cuda()
    e, c = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    J = gpu_rc(ctx, nx, nz, eg, cg, W, 2, 1e30, 3, 8, [0, 1, 2], i_bc=0.7, log_mean=True)
    Jr, probes = oracle_rc(e, c, W, 2, 1e30, 3, 8, [0, 1, 2], i_bc=0.7, mean="log")
    assert_rel(J[:, probes], Jr[:, probes], what="J")


def test_rc_paper_configuration(ctx):
    nx, nz, L = 128, 128, 8
    eg, cg, e, c = line2(ctx, nx, nz, L, synth.SEED_BASE + 430)
    caps = [0, 0, 1, 2, 3, 3]
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 3, 1e30, 6, 4, caps)
    Jr, probes = oracle_rc(e, c, 8, 3, 1e30, 6, 4, caps)
    assert_rel(J[:, probes], Jr[:, probes], what="J")


def _bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def test_rc_bf16_bricks_level0(ctx):
    nx, nz, L = 64, 64, 8
    eg, cg, e, c = line2(ctx, nx, nz, L, synth.SEED_BASE + 440)
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 0, 1e30, 3, 4, [0, 0, 0], storage=1)
    e32, c32 = e.astype(np.float32), c.astype(np.float32)
    S = np.where(c32 > 0, e32 / np.where(c32 > 0, c32, 1), 0).astype(np.float32)
    Sb, cb = _bf16(S).astype(np.float64), _bf16(c32).astype(np.float64)
    Jr, probes = oracle_rc(Sb * cb, cb, 8, 0, 1e30, 3, 4, [0, 0, 0])
    assert_rel(J[:, probes], Jr[:, probes], what="J")


def test_rc_paper_configuration_512(ctx):
    # the cascade report's configuration (6 cascades, caps [0, 0, 1, 2, 3, 3], VLM 0-3)
    # on a 512^2 instance of its workload, every probe of every non-empty block
    nx = nz = 512
    L = 8
    eg, cg, e, c = line2(ctx, nx, nz, L, synth.SEED_BASE + 450)
    caps = [0, 0, 1, 2, 3, 3]
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 3, 1e30, 6, 4, caps)
    Jr, probes = oracle_rc(e, c, 8, 3, 1e30, 6, 4, caps)
    assert_rel(J[:, probes], Jr[:, probes], what="J")


def test_rc_bench_configuration_1024(ctx):
    # the benchmark's cascade section at full size: its 1024^2 atmosphere (one
    # batch of 8 wavelengths), 6 cascades, caps [0, 0, 1, 2, 3, 3], VLM 0-3 with
    # unlimited averaging (no level decision near a threshold), every probe
    nx = nz = 1024
    eg, cg, e, c = line2(ctx, nx, nz, 8, synth.SEED_BASE + 2)
    caps = [0, 0, 1, 2, 3, 3]
    J = gpu_rc(ctx, nx, nz, eg, cg, 8, 3, 1e30, 6, 4, caps)
    Jr, probes = oracle_rc(e, c, 8, 3, 1e30, 6, 4, caps)
    assert_rel(J[:, probes], Jr[:, probes], what="J")
