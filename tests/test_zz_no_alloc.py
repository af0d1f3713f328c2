"""The allocation-free batched solve (dex_batch_solve_noalloc).

Some callers cannot allocate device memory when they solve -- a host application
that owns the device through its own memory pool, or a time-critical loop that
cannot afford cudaMalloc's possible device synchronisation.  For them the library
keeps the batched solve's one scratch word (its work counter) in a static device
array.  This test calls that entry point through the C ABI twice in a row (the
second call reuses the array the first one left behind) and checks both results
against the ordinary dex_batch_solve, which takes its counter from the caller.
The two run the same kernel in the same order, so the results must be identical.
Around the second call it also checks that the device's free memory
(cudaMemGetInfo) and torch's allocation count do not change.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [dict(nx=64, nz=48, n_lambda=16, n_dir=8, empty_frac=0.3, seed=21),
         dict(nx=96, nz=64, n_lambda=24, n_dir=12, empty_frac=0.5, seed=22),
         dict(nx=48, nz=96, n_lambda=8, n_dir=16, empty_frac=0.1, seed=23)]


def _atmospheres(ctx, api):
    out = []
    for sp in SPECS:
        m = synth.sparse_line_atmosphere(sp["nx"], sp["nz"], n_lambda=sp["n_lambda"], empty_frac=sp["empty_frac"],
                                         seed=sp["seed"])
        t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
             for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
        eta, chi = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
        grid = api.grid_build(ctx, sp["nx"], sp["nz"], eta, chi)
        mips = api.mips_build(ctx, grid, eta, chi, 8, 3, 1.0, 1.0, 0.25)
        dirs, w = synth.directions(sp["n_dir"])
        out.append(dict(grid=grid, mips=mips, dirs=torch.from_numpy(dirs).cuda(), w=torch.from_numpy(w).cuda(),
                        J=torch.empty((sp["n_lambda"], sp["nx"] * sp["nz"]), device="cuda")))
    return out


def test_noalloc_batch_matches_batch_solve_twice():
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    atms = _atmospheres(ctx, api)
    band = [6.0, 24.0, 96.0]
    items = [api.batch_item(a["grid"], a["mips"], a["dirs"], a["w"], a["J"], band=band) for a in atms]
    api.batch_solve(ctx, items, 8)                       # caller-provided work counter
    ctx.check()
    ref = [a["J"].clone() for a in atms]
    done = torch.zeros(len(atms), dtype=torch.int64, device="cuda")
    start = torch.zeros(1, dtype=torch.int64, device="cuda")
    for call in range(2):                                # the second call reuses the static scratch
        for a in atms:
            a["J"].fill_(-1.0)
        torch.cuda.synchronize()
        # after the first call (which may make the driver load the library's kernels)
        # the call must change neither the device's free memory nor torch's allocations
        free0, n_alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        api.batch_solve_noalloc(ctx, items, 8, done_ns=done, start_ns=start)
        ctx.check()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed during the call"
            assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == n_alloc0
        for a, r in zip(atms, ref):
            assert torch.equal(a["J"], r), f"call {call}: result differs from dex_batch_solve"
        assert (done.cpu().numpy() >= int(start.item())).all()
