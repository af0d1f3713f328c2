"""Population-workload report: the Lambda iteration at full size on the GPU.

Runs the three-level-atom iteration (96 wavelengths, 96 directions, 20 steps
from LTE) on an n x n seeded atmosphere with the plain full-resolution solve
and with the accelerated solve (VLM levels 0-3, distance limits) for several
IoD thresholds and brick storage formats, and reports the time per iteration
and the population error of each accelerated run against the plain one (the
plain float32 path agrees with the float64 oracle to ~1e-5 on the reduced
instance of the tests).  Every step is a library call; this module only
sequences them.

With ``--cascades`` the formal solution is the radiance-cascade solve (6
cascades, 4 cascade-0 directions, interval end 1.5; the paper's solver): full
resolution as the reference, then VLM levels 0-3 with the per-cascade caps
[0, 0, 1, 2, 3, 3] at IoD 1e-2, 1 and unlimited averaging.

Usage: python -m paper_2511_08498_gb300.populations [--n 1024] [--iters 20] [--cascades]
       [--walk paired|per_batch] [--out FILE]
"""

from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

from . import api

BAND = [6.0, 24.0, 96.0]
RUNS = [(1e-2, api.STORE_F32), (1e-2, api.STORE_F16), (1e-2, api.STORE_BF16), (1.0, api.STORE_F32),
        (1.0, api.STORE_F16), (1e30, api.STORE_F32)]


RC = {"n_cascades": 6, "n0": 4, "t0": 1.5, "level_cap": [0, 0, 1, 2, 3, 3]}
RC_RUNS = [(1e-2, api.STORE_F32), (1.0, api.STORE_F32), (1e30, api.STORE_F32)]


def report(n=1024, n_iter=20, n_dir=96, cascades=False, walk="paired"):
    import synth
    from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom
    ctx = api.Context(0)
    ad = three_level_atom()
    m = populations_atmosphere(n, n, seed=synth.SEED_BASE + 4)
    lam, tag = line_wavelength_grid()
    dirs, w = synth.directions(n_dir)
    atom = api.Atom.from_dict(ad, m["cell_cm"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in ("temperature", "ne", "nh")}
    live = torch.from_numpy(m["temperature"].reshape(-1) > 0).cuda()

    # the accelerated long-characteristics runs walk once per mirror pair of a
    # line's wavelength batches when each line's samples fill whole batches of 8
    n_per_line = int(np.sum(tag == 0))
    group = n_per_line // 8 if n_per_line % 8 == 0 else 0
    paired = walk == "paired" and not cascades
    ctx.set_traversal(api.TRAVERSAL_PAIRED if paired else api.TRAVERSAL_PER_BATCH)
    ctx.set_pair_group(group if paired else 0)

    def run(accelerated, iod=1e-2, storage=api.STORE_F32):
        torch.cuda.synchronize()
        t0 = time.time()
        p = api.lambda_iteration(ctx, atom, lam, tag, dev["temperature"], dev["ne"], dev["nh"], n, n, dirs, w,
                                 n_iter, accelerated=accelerated, iod=iod, band=BAND, storage=storage,
                                 cascades=RC if cascades else None)
        ctx.check()
        return p, (time.time() - t0) / n_iter

    ref, t_plain = run(False)
    solver = (f"radiance cascades {RC}" if cascades else
              f"long characteristics, {n_dir} directions, distance limits {BAND}, " +
              (f"one walk per mirror pair of a line's wavelength batches (pair group {group})" if paired else
               "one walk per wavelength batch"))
    out = {"workload": f"three-level atom, {n}x{n}, {lam.size} wavelengths, {n_iter} Lambda steps from LTE, "
                       f"VLM mip 0-3; formal solution: {solver}",
           "plain": {"s_per_iteration": t_plain}, "accelerated": []}
    for iod, storage in (RC_RUNS if cascades else RUNS):
        p, t = run(True, iod, storage)
        e = ((p - ref).abs() / ref.abs().clamp_min(1e-300))[:, live].reshape(-1).double().cpu().numpy() * 100.0
        out["accelerated"].append({"iod": iod, "storage": ["f32", "bf16", "f16"][storage], "s_per_iteration": t,
                                   "speedup_vs_plain": t_plain / t,
                                   "pop_err_pct_vs_plain": {q: float(np.percentile(e, v)) for q, v in
                                                            (("p50", 50), ("p99", 99), ("p99.9", 99.9),
                                                             ("max", 100))}})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--cascades", action="store_true")
    ap.add_argument("--walk", default="paired", choices=["paired", "per_batch"],
                    help="walk of the accelerated long-characteristics runs")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    rep = report(args.n, args.iters, cascades=args.cascades, walk=args.walk)
    s = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    sys.exit(main())
