"""Moving-medium report: the treatments of Section 3 on one seeded atmosphere.

Runs, on a 2048 x 1024 moving-medium atmosphere (64 wavelengths, 64 directions
by default):
  * the Core-and-Voigt solve at full resolution (MIP 0 only, every probe of
    every non-empty block): the exact-profile reference of this report;
  * Core and Voigt with VLM levels 0-3 and distance limits, and velocity
    interpolation (8 stored velocity samples) with the same levels, each with
    three level tests: the paper's (IoD plus the always-average rule for
    chi Ds < 0.25), the IoD test alone, and the IoD test alone plus the test in
    8 propagation directions;
  * optionally Core and Voigt with the learned profile (``--mlp PARAMS.npy``),
    on a reduced atmosphere because it evaluates the network per segment.
Each is timed with CUDA events; J is compared with the reference (relative
error percentiles over every probe and wavelength with J > 0), and the
dense-equivalent throughput (MIP-0 segment-wavelengths of the reference) is
reported.  Every step is a library call; this module only sequences them.

Usage: python -m paper_2511_08498_gb300.moving [--nx 2048 --nz 1024] [--out FILE]
"""

from __future__ import annotations

import argparse
import json
import sys

import numpy as np
import torch

from . import api

BAND = [6.0, 24.0, 96.0]


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


def _err(J, ref):
    mask = ref > 0
    e = ((J - ref).abs() / ref.clamp_min(1e-30))[mask].double().cpu().numpy() * 100.0
    return {"p50": float(np.median(e)), "p99": float(np.quantile(e, 0.99)), "p99.9": float(np.quantile(e, 0.999)),
            "max": float(e.max())}


def dense_seg_lambda(ctx, grid, n_lambda, W, dirs, w):
    """Full-resolution segment-wavelengths of every probe (every cell of every
    non-empty block) over all directions: the plain solver's counting pass, which
    walks every cell whatever the medium (zero planes suffice)."""
    act = torch.nonzero(grid.block_offset >= 0).reshape(-1)
    bx, bz = act % grid.nbx, act // grid.nbx
    loc = torch.arange(256, device=act.device)
    cells = ((bz[:, None] * 16 + loc[None, :] // 16) * grid.nx + bx[:, None] * 16 + loc[None, :] % 16)
    cells = cells.reshape(-1).to(torch.int32)
    planes = torch.zeros((1, grid.nx * grid.nz, 2 * W), device="cuda")
    _, _, seg = api.formal_solve_dense(ctx, grid.nx, grid.nz, W, W, planes, dirs, w, probes=cells,
                                       count_segments=True)
    ctx.check()
    return int(seg.item()) * -(-n_lambda // W) * W


# level-test variants: (name suffix, always-average threshold chi_ds_min, directional tests K)
LEVEL_TESTS = (("", 0.25, 0), ("_iod_only", 0.0, 0), ("_iod_only_dirtest8", 0.0, 8))


def report(nx=2048, nz=1024, n_lambda=64, n_dir=64, W=8, max_mip=3, iod=1e-2, mlp_params=None, mlp_nx=256,
           mlp_nz=128, reps=2, level_tests=LEVEL_TESTS):
    import synth
    ctx = api.Context(0)
    m = synth.dynamic_line_atmosphere(nx, nz, n_lambda=n_lambda, seed=synth.SEED_BASE + 3)
    f = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in api.CAV_FIELDS}
    dirs, w = synth.directions(n_dir)
    grid = api.cav_grid_build(ctx, nx, nz, f)
    n_cells = nx * nz
    ref = torch.empty((n_lambda, n_cells), device="cuda")
    plain = api.cav_mips_build(ctx, grid, f, m["dv"], m["c_kms"], W, 0, iod, iod, 0.25)
    dense = dense_seg_lambda(ctx, grid, n_lambda, W, dirs, w)
    t_plain = _time(lambda: api.formal_solve_cav(ctx, grid, plain, dirs, w, J=ref), reps)
    out = {"workload": f"moving-medium atmosphere {nx}x{nz}, {n_lambda} wavelengths, {n_dir} directions, "
                       f"W={W}, VLM mip 0-{max_mip}, IoD {iod:g}, distance limits {BAND}",
           "dense_seg_lambda": dense,
           "cav_plain": {"ms": t_plain * 1e3, "seg_lambda_per_s": dense / t_plain}}
    Jc = torch.empty_like(ref)
    Jv = torch.empty_like(ref)
    # velocity interpolation at full resolution: the error of interpolating the
    # profile between the stored velocity samples, before any mipmapping
    vel0 = api.vel_mips_build(ctx, grid, f, m["dv"], m["c_kms"], W, 0, iod, iod, 0.25)
    t_vel0 = _time(lambda: api.formal_solve_velinterp(ctx, grid, vel0, dirs, w, J=Jv), reps)
    ctx.check()
    out["velinterp_mip0"] = {"ms": t_vel0 * 1e3, "speedup_vs_plain": t_plain / t_vel0,
                             "j_err_pct_vs_plain": _err(Jv, ref)}
    for tag, cm, K in level_tests:
        cav = api.cav_mips_build(ctx, grid, f, m["dv"], m["c_kms"], W, max_mip, iod, iod, cm, test_dirs=K)
        t_cav = _time(lambda: api.formal_solve_cav(ctx, grid, cav, dirs, w, J=Jc, band=BAND), reps)
        _, _, sc = api.formal_solve_cav(ctx, grid, cav, dirs, w, J=Jc, band=BAND, count_segments=True)
        ctx.check()
        lt = {"chi_ds_min": cm, "directional_tests": K}
        out["cav_vlm" + tag] = {"ms": t_cav * 1e3, "seg_lambda_per_s": dense / t_cav,
                                "speedup_vs_plain": t_plain / t_cav, "executed_fraction": int(sc.item()) * W / dense,
                                "level_test": lt, "j_err_pct_vs_plain": _err(Jc, ref)}
        vel = api.vel_mips_build(ctx, grid, f, m["dv"], m["c_kms"], W, max_mip, iod, iod, cm, test_dirs=K)
        t_vel = _time(lambda: api.formal_solve_velinterp(ctx, grid, vel, dirs, w, J=Jv, band=BAND), reps)
        ctx.check()
        out["velinterp_vlm" + tag] = {"ms": t_vel * 1e3, "seg_lambda_per_s": dense / t_vel,
                                      "speedup_vs_plain": t_plain / t_vel, "level_test": lt,
                                      "j_err_pct_vs_plain": _err(Jv, ref)}
    if mlp_params is not None:
        ms = synth.dynamic_line_atmosphere(mlp_nx, mlp_nz, n_lambda=n_lambda, seed=synth.SEED_BASE + 3)
        fs = {k: torch.from_numpy(np.ascontiguousarray(ms[k]).reshape(-1)).cuda() for k in api.CAV_FIELDS}
        gs = api.cav_grid_build(ctx, mlp_nx, mlp_nz, fs)
        cs = api.cav_mips_build(ctx, gs, fs, ms["dv"], ms["c_kms"], W, max_mip, iod, iod, 0.25)
        J0 = torch.empty((n_lambda, mlp_nx * mlp_nz), device="cuda")
        J1 = torch.empty_like(J0)
        t0 = _time(lambda: api.formal_solve_cav(ctx, gs, cs, dirs, w, J=J0, band=BAND), reps)
        t1 = _time(lambda: api.formal_solve_cav(ctx, gs, cs, dirs, w, J=J1, band=BAND, mlp_params=mlp_params), 1)
        ctx.check()
        out["cav_mlp_reduced"] = {"grid": [mlp_nx, mlp_nz], "cav_ms": t0 * 1e3, "cav_mlp_ms": t1 * 1e3,
                                  "slowdown": t1 / t0, "j_err_pct_vs_cav": _err(J1, J0)}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--nz", type=int, default=1024)
    ap.add_argument("--iod", type=float, default=1e-2)
    ap.add_argument("--mlp", default=None, help="surrogate parameters (.npy, 4481 floats)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    mlp = None if args.mlp is None else np.load(args.mlp)
    rep = report(args.nx, args.nz, iod=args.iod, mlp_params=mlp)
    s = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    sys.exit(main())
