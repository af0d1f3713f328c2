"""Train the learned Voigt-profile surrogate and report what it gains.

Steps (each a library call; this module only sequences them):
  1. draw 2^k sample points (x, a, u) over the moving-medium workload's ranges,
     half of them concentrated on the line core (synth.mlp.voigt_samples);
  2. targets ln H(a, x - u) from the library's own Voigt evaluation (dex_mlp_targets);
  3. minibatch Adam on the tensor-core gradient kernel (dex_mlp_grad, dex_mlp_adam);
  4. evaluate on held-out uniform samples against the same exact-profile evaluation:
     relative error of H, and evaluation throughput of the network (tcgen05
     inference, dex_mlp_forward) against the Voigt kernel (dex_voigt);
  5. the Core-and-Voigt solve of a moving-medium atmosphere with the exact
     profile and with the network (dex_formal_solve_cav / _cav_mlp): time and
     relative J difference.

Usage: python -m paper_2511_08498_gb300.surrogate [--log2-samples 24] [--steps N] [--out FILE]
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

from . import api


def _time(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def train(ctx, log2_samples=24, steps=20000, batch=16384, lr=3e-3, lr_final=3e-5, seed_offset=0,
          core_fraction=0.5):
    import synth
    n = 1 << log2_samples
    xau = torch.from_numpy(synth.mlp.voigt_samples(n, seed=synth.SEED_BASE + 970 + seed_offset,
                                                   core_fraction=core_fraction)).cuda()
    target = api.mlp_targets(ctx, xau)
    params = torch.from_numpy(synth.mlp.initial_params()).cuda()
    t0 = time.time()
    losses = api.mlp_train(ctx, xau, target, params, steps=steps, batch=batch, lr=lr, lr_final=lr_final,
                           log_every=max(1, steps // 20))
    ctx.check()
    return params, losses, time.time() - t0


def evaluate(ctx, params, n_held=1 << 16, n_time=1 << 22):
    import synth
    held = torch.from_numpy(synth.mlp.voigt_samples(n_held, seed=synth.SEED_BASE + 980)).cuda()
    y = api.mlp_forward(ctx, held, params)
    a = held[:, 1].contiguous()
    xs = (held[:, 0] - held[:, 2]).contiguous()
    h = api.voigt(ctx, a, xs)
    err = (torch.exp(y.double()) - h.double()).abs() / h.double()
    e = err.cpu().numpy()
    big = torch.from_numpy(synth.mlp.voigt_samples(n_time, seed=synth.SEED_BASE + 981)).cuda()
    out = torch.empty(n_time, device="cuda")
    ab, xb = big[:, 1].contiguous(), (big[:, 0] - big[:, 2]).contiguous()
    t_mlp = _time(lambda: api.mlp_forward(ctx, big, params, out=out))
    t_vgt = _time(lambda: api.voigt(ctx, ab, xb, out=out))
    ctx.check()
    return {"held_out_samples": n_held,
            "rel_err_H_vs_library_voigt": {"p50": float(np.median(e)), "p90": float(np.quantile(e, 0.9)),
                                           "p99": float(np.quantile(e, 0.99)), "max": float(e.max())},
            "throughput_per_s": {"mlp_tcgen05": n_time / t_mlp, "voigt_hum1wei24": n_time / t_vgt},
            "mlp_flop_per_eval": 2 * (3 * 64 + 64 * 64 + 64)}


def cav_compare(ctx, params, nx=256, nz=128, n_lambda=64, n_dir=64, max_mip=3, band=(6.0, 24.0, 96.0)):
    import synth
    m = synth.dynamic_line_atmosphere(nx, nz, n_lambda=n_lambda, seed=synth.SEED_BASE + 990)
    f = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in api.CAV_FIELDS}
    dirs, w = synth.directions(n_dir)
    grid = api.cav_grid_build(ctx, nx, nz, f)
    mp = api.cav_mips_build(ctx, grid, f, m["dv"], m["c_kms"], 8, max_mip, 1.0, 1.0, 0.25)
    J0 = torch.empty((n_lambda, nx * nz), device="cuda")
    J1 = torch.empty_like(J0)
    host = params.cpu().numpy()
    t_exact = _time(lambda: api.formal_solve_cav(ctx, grid, mp, dirs, w, band=list(band), J=J0), reps=2)
    t_mlp = _time(lambda: api.formal_solve_cav(ctx, grid, mp, dirs, w, band=list(band), J=J1, mlp_params=host),
                  reps=1)
    ctx.check()
    mask = J0 > 0
    e = ((J1 - J0).abs() / J0.clamp_min(1e-30))[mask].double().cpu().numpy()
    return {"workload": f"moving-medium atmosphere {nx}x{nz}, {n_lambda} wavelengths, {n_dir} directions, "
                        f"VLM mip 0-{max_mip}, IoD 1, distance limits {list(band)}",
            "cav_exact_ms": t_exact * 1e3, "cav_mlp_ms": t_mlp * 1e3, "slowdown": t_mlp / t_exact,
            "J_rel_diff_mlp_vs_exact": {"p50": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
                                        "p99.9": float(np.quantile(e, 0.999)), "max": float(e.max())}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2-samples", type=int, default=24)
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--lr-final", type=float, default=3e-5)
    ap.add_argument("--core-fraction", type=float, default=0.5)
    ap.add_argument("--out", default=None)
    ap.add_argument("--no-cav", action="store_true")
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    args = ap.parse_args(argv)
    ctx = api.Context(0)
    params, losses, secs = train(ctx, args.log2_samples, args.steps, args.batch, args.lr, args.lr_final,
                                 core_fraction=args.core_fraction)
    rep = {"samples": 1 << args.log2_samples, "steps": args.steps, "batch": args.batch, "lr": args.lr,
           "lr_final": args.lr_final, "core_fraction": args.core_fraction, "train_seconds": secs,
           "loss_curve": losses}
    if args.save:
        np.save(args.save, params.cpu().numpy())
    rep.update(evaluate(ctx, params))
    if not args.no_cav:
        rep["cav"] = cav_compare(ctx, params)
    s = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    sys.exit(main())
