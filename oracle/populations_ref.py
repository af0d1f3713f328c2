"""Write the float64 oracle's level populations for the population workload at a
reduced size (test infrastructure: the stored values the GPU population test
compares with).

The workload is the three-level-atom Lambda iteration (2 lines x 40 samples +
16 continuum samples = 96 wavelengths, 96 directions, 20 fixed steps from LTE)
on a seeded stratified atmosphere; the formal solution is the plain float64
long-characteristics oracle at full resolution from every cell of every
non-empty block.  Everything in float64 (no float32 rounding of the
emissivity/opacity), so the stored populations are the reference the GPU's
float32 path and its reduced-precision storage are compared with.

Usage: python -m oracle.populations_ref [--n 128] [--out tests/golden/populations_128.npz]
"""

from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ITER = 20
N_DIR = 96


def populations(n: int, n_iter: int = N_ITER, n_dir: int = N_DIR):
    import synth
    from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom

    from . import atom as oa
    from . import lc
    from . import mips as omips
    ad = three_level_atom()
    m = populations_atmosphere(n, n, seed=synth.SEED_BASE + 4)
    lam, tag = line_wavelength_grid()
    dirs, w = synth.directions(n_dir)
    T, ne, nh = (m[k].astype(np.float64) for k in ("temperature", "ne", "nh"))
    pops = oa.lte_populations(ad, T, nh)
    for _ in range(n_iter):
        eta, chi = oa.eta_chi(ad, lam, tag, T, ne, pops, m["cell_cm"])
        empty = omips.block_empty(eta, chi, 16)
        probes = omips.probes_of_blocks(empty, 16)
        Jp = lc.formal_solve(eta, chi, dirs, w, probes=probes)
        J = np.zeros((lam.size, n * n))
        J[:, probes] = Jp
        jb = oa.jbar(ad, lam, tag, T.reshape(-1), J)
        pops = oa.se_solve(ad, T.reshape(-1), ne.reshape(-1), nh.reshape(-1), jb).reshape((3,) + T.shape)
    return pops.reshape(3, -1)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    out = args.out or os.path.join(ROOT, "tests", "golden", f"populations_{args.n}.npz")
    t0 = time.time()
    p = populations(args.n)
    np.savez_compressed(out, populations=p, n=args.n, n_iter=N_ITER, n_dir=N_DIR,
                        seed_offset=4, note="float64 oracle, plain Lambda iteration from LTE")
    print(f"wrote {out} ({time.time() - t0:.1f} s)")


if __name__ == "__main__":
    sys.exit(main())
