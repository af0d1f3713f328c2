"""Radiance-cascade report: the cascade solver on the static line workload.

Runs, on the seeded 1024 x 1024 sparse static line atmosphere (32 wavelengths,
16^2 blocks, W = 8; the long-characteristics benchmark's input):
  * the radiance-cascade solve at full resolution (MIP 0 only), the paper's
    configuration otherwise (6 cascades, 4 cascade-0 directions, interval end
    1.5 voxels): the reference of this report;
  * the same with VLM levels and the per-cascade level caps [0, 0, 1, 2, 3, 3]
    (the paper's [0, 0, 1, 2, 3, 4] within levels 0-3) at each IoD threshold;
  * the long-characteristics solve (64 directions, full resolution) for scale,
    with the relative difference of the cascade J from it (the cascades'
    angular and spatial interpolation, not an error of the acceleration).
Each solve is timed with CUDA events (the whole cascade hierarchy and the J
reduction); the executed segment-wavelengths and their rate against the
measured 2^x throughput are reported.  Every step is a library call.

Usage: python -m paper_2511_08498_gb300.cascades [--n 1024] [--iod 1e-2 1 1e30] [--out FILE]
"""

from __future__ import annotations

import argparse
import json
import sys

import numpy as np
import torch

from . import api

N_CASCADES, N0, T0 = 6, 4, 1.5
CAPS = [0, 0, 1, 2, 3, 3]


def _time(fn, reps=2):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def _diff(J, ref, mask):
    m = mask & (ref > 0)
    e = ((J - ref).abs() / ref.clamp_min(1e-30))[m].double().cpu().numpy() * 100.0
    return {"p50": float(np.median(e)), "p99": float(np.quantile(e, 0.99)), "p99.9": float(np.quantile(e, 0.999)),
            "max": float(e.max())}


def report(n=1024, n_lambda=32, W=8, max_mip=3, iods=(1e-2, 1.0, 1e30), reps=2):
    import synth
    ctx = api.Context(0)
    m = synth.sparse_line_atmosphere(n, n, n_lambda=n_lambda, seed=synth.SEED_BASE + 2)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eta, chi = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    grid = api.grid_build(ctx, n, n, eta, chi)
    active = (grid.block_offset.view(grid.nbz, grid.nbx) >= 0)
    mask = active.repeat_interleave(16, 0).repeat_interleave(16, 1).reshape(1, -1).expand(n_lambda, -1)
    peak = api.measure_ex2_rate(ctx)
    ws = torch.empty(api.rc_workspace_floats(n, n, n_lambda, W, N0), device="cuda")
    out = {"workload": f"static line atmosphere {n}x{n}, {n_lambda} wavelengths, W={W}; radiance cascades: "
                       f"{N_CASCADES} cascades, {N0} cascade-0 directions, t0 {T0}, caps {CAPS}",
           "ex2_per_s": peak}

    def run(mp, caps, J):
        return api.rc_solve(ctx, grid, mp, N_CASCADES, N0, T0, level_cap=caps, J=J, workspace=ws)

    def measured(mp, caps, J):
        t_s = _time(lambda: run(mp, caps, J), reps)
        _, seg = api.rc_solve(ctx, grid, mp, N_CASCADES, N0, T0, level_cap=caps, J=J, workspace=ws,
                              count_segments=True)
        ctx.check()
        executed = int(seg.item()) * W
        return t_s, executed

    ref = torch.empty((n_lambda, n * n), device="cuda")
    mp0 = api.mips_build(ctx, grid, eta, chi, W, 0, 1e30, 1e30, 0.25)
    t0_, ex0 = measured(mp0, [0] * N_CASCADES, ref)
    out["rc_full_resolution"] = {"ms": t0_ * 1e3, "executed_seg_lambda": ex0,
                                 "seg_lambda_per_s": ex0 / t0_, "ex2_frac": ex0 / t0_ / peak}
    del mp0
    # long characteristics, 64 directions, full resolution, for scale
    dirs, w = synth.directions(64)
    planes = api.pack_planes(ctx, eta, chi, W)
    probes = torch.nonzero(mask[0]).reshape(-1).to(torch.int32)
    Jlc_p = torch.empty((n_lambda, probes.numel()), device="cuda")
    t_lc = _time(lambda: api.formal_solve_dense(ctx, n, n, n_lambda, W, planes, dirs, w, probes=probes, J=Jlc_p), reps)
    ctx.check()
    del planes
    Jlc = torch.zeros_like(ref)
    Jlc[:, probes.long()] = Jlc_p
    out["lc_64_directions"] = {"ms": t_lc * 1e3, "rc_full_resolution_diff_pct": _diff(ref, Jlc, mask)}
    J = torch.empty_like(ref)
    for iod in iods:
        mp = api.mips_build(ctx, grid, eta, chi, W, max_mip, iod, iod, 0.25)
        t_a, ex = measured(mp, CAPS, J)
        lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
        out[f"rc_vlm_iod_{iod:g}"] = {
            "ms": t_a * 1e3, "speedup_vs_full_resolution": t0_ / t_a, "executed_seg_lambda": ex,
            "executed_fraction": ex / ex0, "ex2_frac": ex / t_a / peak,
            "level_counts": {str(L): int((lev == L).sum()) for L in range(-1, max_mip + 1)},
            "j_err_pct_vs_full_resolution": _diff(J, ref, mask)}
        del mp
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--iod", type=float, nargs="+", default=[1e-2, 1.0, 1e30])
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    rep = report(args.n, iods=tuple(args.iod))
    s = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    sys.exit(main())
