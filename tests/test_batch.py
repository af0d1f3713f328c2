"""Batched persistent solve: bit-identical to per-atmosphere solves (same traversal,
same summation order), and to the oracle through them."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def build_atmospheres(ctx, specs, W=8, iod=1.0, band=(6.0, 24.0, 96.0)):
    from paper_2511_08498_gb300 import api
    out = []
    for sp in specs:
        m = synth.sparse_line_atmosphere(sp["nx"], sp["nz"], n_lambda=sp["n_lambda"], empty_frac=sp["empty_frac"],
                                         seed=sp["seed"])
        t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
             for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
        eta, chi = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
        grid = api.grid_build(ctx, sp["nx"], sp["nz"], eta, chi)
        mp = api.mips_build(ctx, grid, eta, chi, W, 3, iod, iod, 0.25)
        dirs, w = synth.directions(sp["n_dir"])
        out.append(dict(grid=grid, mips=mp, dirs=dirs, w=w, dirs_dev=torch.from_numpy(dirs).cuda(),
                        w_dev=torch.from_numpy(w).cuda(), band=list(band),
                        J=torch.empty((sp["n_lambda"], sp["nx"] * sp["nz"]), device="cuda")))
    return out


SPECS = [dict(nx=64, nz=48, n_lambda=16, n_dir=8, empty_frac=0.3, seed=11),
         dict(nx=96, nz=64, n_lambda=24, n_dir=12, empty_frac=0.5, seed=12),
         dict(nx=48, nz=96, n_lambda=8, n_dir=16, empty_frac=0.1, seed=13),
         dict(nx=128, nz=32, n_lambda=8, n_dir=4, empty_frac=0.7, seed=14)]


@pytest.mark.parametrize("ctas", [0, 1, 7])
def test_batch_equals_per_atmosphere(ctas):
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    atms = build_atmospheres(ctx, SPECS)
    refs = []
    for a in atms:
        J, _, _ = api.formal_solve_hdda(ctx, a["grid"], a["mips"], a["dirs"], a["w"], band=a["band"])
        refs.append(J.clone())
    items = [api.batch_item(a["grid"], a["mips"], a["dirs_dev"], a["w_dev"], a["J"], band=a["band"]) for a in atms]
    done, start = api.batch_solve(ctx, items, 8, ctas=ctas, timing=True)
    ctx.check()
    for a, r in zip(atms, refs):
        assert torch.equal(a["J"], r)
    d = done.cpu().numpy()
    assert (d > 0).all() and (d >= int(start.item())).all()


# every knob of the batched launch the autotuner sweeps: probes per work item,
# items per queue claim, block-table staging, register budget, grid size
CONFIGS = [dict(ctas=0, packet=128, chunk=1, staging=0, occupancy=0),
           dict(ctas=5, packet=64, chunk=3, staging=1, occupancy=0),
           dict(ctas=0, packet=256, chunk=8, staging=1, occupancy=1),
           dict(ctas=304, packet=64, chunk=2, staging=0, occupancy=1),
           dict(ctas=1, packet=128, chunk=64, staging=1, occupancy=1)]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_every_configuration_equals_per_atmosphere(cfg):
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    atms = build_atmospheres(ctx, SPECS)
    refs = []
    for a in atms:
        J, _, _ = api.formal_solve_hdda(ctx, a["grid"], a["mips"], a["dirs"], a["w"], band=a["band"])
        refs.append(J.clone())
    items = [api.batch_item(a["grid"], a["mips"], a["dirs_dev"], a["w_dev"], a["J"], band=a["band"]) for a in atms]
    for a in atms:
        a["J"].fill_(-1.0)
    done, start = api.batch_solve_config(ctx, items, 8, timing=True, **cfg)
    ctx.check()
    for a, r in zip(atms, refs):
        assert torch.equal(a["J"], r), cfg
    d = done.cpu().numpy()
    assert (d > 0).all() and (d >= int(start.item())).all()


def test_configuration_is_checked():
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    atms = build_atmospheres(ctx, SPECS[:1])
    items = [api.batch_item(a["grid"], a["mips"], a["dirs_dev"], a["w_dev"], a["J"], band=a["band"]) for a in atms]
    for bad in (dict(packet=96), dict(chunk=0), dict(chunk=65), dict(staging=2), dict(occupancy=3)):
        with pytest.raises(api.DexError):
            api.batch_solve_config(ctx, items, 8, **bad)


# the paired walk (DEX_TRAVERSAL_PAIRED): work units are the pairs of batches and
# the lone batches; 16, 24 and 8 wavelengths give one pair, one pair and a lone
# batch, and a lone batch; pair group 2 pairs 0-1 of the 24-wavelength atmosphere
# and leaves batch 2 alone
@pytest.mark.parametrize("cfg,group", [(dict(ctas=0, packet=256, chunk=1, staging=0, occupancy=0), 0),
                                       (dict(ctas=7, packet=128, chunk=3, staging=1, occupancy=1), 0),
                                       (dict(ctas=0, packet=64, chunk=2, staging=0, occupancy=0), 2)])
def test_paired_batch_equals_per_atmosphere_paired_solves(cfg, group):
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    atms = build_atmospheres(ctx, SPECS)
    ctx.set_traversal(api.TRAVERSAL_PAIRED)
    ctx.set_pair_group(group)
    try:
        refs = []
        for a in atms:
            J, _, _ = api.formal_solve_hdda(ctx, a["grid"], a["mips"], a["dirs"], a["w"], band=a["band"])
            refs.append(J.clone())
        items = [api.batch_item(a["grid"], a["mips"], a["dirs_dev"], a["w_dev"], a["J"], band=a["band"])
                 for a in atms]
        for a in atms:
            a["J"].fill_(-1.0)
        done, start = api.batch_solve_config(ctx, items, 8, timing=True, **cfg)
        ctx.check()
    finally:
        ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
        ctx.set_pair_group(0)
    for a, r in zip(atms, refs):
        assert torch.equal(a["J"], r), cfg
    d = done.cpu().numpy()
    assert (d > 0).all() and (d >= int(start.item())).all()
