"""3D report: the plain and the accelerated formal solution on a 3D atmosphere.

Runs, on a seeded 3D sparse line atmosphere (256^3 cells in 8^3 blocks, 16
wavelengths, a 16-azimuth x 4-inclination quadrature by default):
  * the plain full-resolution 3D solve from every cell of every non-empty block
    (the reference of this report; its counting pass gives the dense-equivalent
    segment-wavelength count the throughputs are normalised by);
  * the accelerated solve (empty-block skipping, VLM levels 0-3, distance
    limits) at each requested IoD threshold, with its MIP-build time, the
    executed-segment fraction, and the relative error of J against the plain
    solve (percentiles over every probe and wavelength with J > 0).
Each solve is timed with CUDA events; the ex2 fraction is executed
segment-wavelength updates per second over the measured 2^x throughput (one
2^x per update).  Every step is a library call; this module only sequences them.

Usage: python -m paper_2511_08498_gb300.grid3d [--n 256] [--iod 1e-2 1.0 1e30] [--out FILE]
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


def block_cells(grid: api.SparseGrid3) -> torch.Tensor:
    """Cell indices of every cell of every active block, block by block in Morton order."""
    n = grid.n_active()
    blk = grid.active[:n].long()
    bx = blk % grid.nbx
    by = (blk // grid.nbx) % grid.nby
    bz = blk // (grid.nbx * grid.nby)
    loc = torch.arange(512, device=blk.device)
    lx, ly, lz = loc % 8, (loc // 8) % 8, loc // 64
    x = bx[:, None] * 8 + lx[None, :]
    y = by[:, None] * 8 + ly[None, :]
    z = bz[:, None] * 8 + lz[None, :]
    return ((z * grid.ny + y) * grid.nx + x).reshape(-1).to(torch.int32)


def workload(n=256, n_lambda=16, seed_offset=31):
    import synth
    ctx = api.Context(0)
    m = synth.sparse_line_atmosphere3(n, n, n, n_lambda=n_lambda, seed=synth.SEED_BASE + seed_offset)
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    eta, chi = api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])
    return ctx, m, eta, chi


def report(n=256, n_lambda=16, n_az=16, n_incl=4, W=8, max_mip=3, iods=(1e-2, 1.0, 1e30), reps=2):
    import synth
    ctx, m, eta, chi = workload(n, n_lambda)
    dirs, w = synth.directions3(n_az, n_incl)
    grid = api.grid3_build(ctx, n, n, n, eta, chi)
    cells = block_cells(grid)
    planes = api.pack_planes(ctx, eta, chi, W)
    _, _, seg = api.formal_solve_dense3(ctx, n, n, n, n_lambda, W, planes, dirs, w, probes=cells,
                                        count_segments=True)
    ctx.check()
    dense = int(seg.item()) * W
    ref = torch.empty((n_lambda, cells.numel()), device="cuda")
    t_plain = _time(lambda: api.formal_solve_dense3(ctx, n, n, n, n_lambda, W, planes, dirs, w, probes=cells, J=ref),
                    reps)
    peak = api.measure_ex2_rate(ctx)
    out = {"workload": f"3D sparse line atmosphere {n}^3 (8^3 blocks, {grid.n_active()} of {grid.n_blocks} "
                       f"active), {n_lambda} wavelengths, {n_az}x{n_incl} directions, W={W}, VLM mip 0-{max_mip}, "
                       f"distance limits {BAND}",
           "dense_seg_lambda": dense, "ex2_per_s": peak,
           "plain": {"ms": t_plain * 1e3, "seg_lambda_per_s": dense / t_plain,
                     "ex2_frac": dense / t_plain / peak}}
    del planes
    J = torch.empty((n_lambda, n ** 3), device="cuda")
    for iod in iods:
        mp = None

        def build():
            nonlocal mp
            mp = api.mips3_build(ctx, grid, eta, chi, W, max_mip, iod, iod, 0.25, out=mp)
        t_build = _time(build, reps)
        lev = api.unpack_states(mp.words.cpu().numpy(), grid.n_blocks)
        # one walk per wavelength batch, and one per mirror pair of batches on the
        # smaller of the pair's levels
        for walk, mode in (("", api.TRAVERSAL_PER_BATCH), ("_paired", api.TRAVERSAL_PAIRED)):
            ctx.set_traversal(mode)
            t_acc = _time(lambda: api.formal_solve_hdda3(ctx, grid, mp, dirs, w, J=J, band=BAND), reps)
            _, _, sc = api.formal_solve_hdda3(ctx, grid, mp, dirs, w, J=J, band=BAND, count_segments=True)
            ctx.check()
            ctx.set_traversal(api.TRAVERSAL_PER_BATCH)
            executed = int(sc.item()) * W
            out[f"vlm_iod_{iod:g}{walk}"] = {
                "ms": t_acc * 1e3, "mips_build_ms": t_build * 1e3, "seg_lambda_per_s": dense / t_acc,
                "speedup_vs_plain": t_plain / t_acc, "executed_fraction": executed / dense,
                "ex2_frac": executed / t_acc / peak,
                "level_counts": {str(L): int((lev == L).sum()) for L in range(-1, max_mip + 1)},
                "j_err_pct_vs_plain": _err(J[:, cells.long()], ref)}
        del mp
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--n-lambda", type=int, default=16)
    ap.add_argument("--iod", type=float, nargs="+", default=[1e-2, 1.0, 1e30])
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    rep = report(args.n, args.n_lambda, iods=tuple(args.iod))
    s = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(s + "\n")
    print(s)


if __name__ == "__main__":
    sys.exit(main())
