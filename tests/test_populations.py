"""Level populations on the GPU vs the float64 oracle.

* LTE start, radiative-rate reduction (float64) and the statistical-equilibrium
  solve (float64): within 1e-10 relative (same inputs; only summation order differs);
* emissivity/opacity from populations (float32 output): within 2e-6 relative;
* a full fixed-length Lambda iteration (20 steps, plain and accelerated paths):
  populations within 1e-4 relative of the oracle's.  Per step the float32 formal
  solution matches to 1e-5 in J; the iteration is a contraction in the optically
  thick lines, so the accumulated population error stays within a few 1e-5.
"""

import numpy as np
import pytest

import synth
from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom
from oracle import atom as oa, lc, mips as omips

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.fixture(scope="module")
def setup():
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    ad = three_level_atom()
    m = populations_atmosphere(48, 48, seed=synth.SEED_BASE + 500)
    lam, tag = line_wavelength_grid(8, 4)
    atom = api.Atom.from_dict(ad, m["cell_cm"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in ("temperature", "ne", "nh")}
    return dict(api=api, ctx=ctx, ad=ad, m=m, lam=lam, tag=tag, atom=atom, dev=dev)


def test_lte_eta_chi_rates_se_units(setup):
    s = setup
    api, ctx, ad, m, dev = s["api"], s["ctx"], s["ad"], s["m"], s["dev"]
    T, ne, nh = m["temperature"], m["ne"], m["nh"]
    live = T.reshape(-1) > 0
    n0 = api.lte_populations(ctx, s["atom"], dev["temperature"], dev["nh"])
    ref0 = oa.lte_populations(ad, T, nh).reshape(3, -1)
    assert rel(n0.cpu().numpy(), ref0)[:, live].max() < 1e-12
    eta, chi = api.atom_eta_chi(ctx, s["atom"], s["lam"], s["tag"], dev["temperature"], dev["ne"], n0)
    er, cr = oa.eta_chi(ad, s["lam"], s["tag"], T, ne, ref0.reshape((3,) + T.shape), m["cell_cm"])
    assert rel(eta.cpu().numpy(), er.reshape(len(s["lam"]), -1)).max() < 2e-6
    assert rel(chi.cpu().numpy(), cr.reshape(len(s["lam"]), -1)).max() < 2e-6
    # rates from a seeded J field (same float32 J on both sides)
    rng = np.random.default_rng(3)
    J = (rng.uniform(0.2, 2.0, (len(s["lam"]), T.size)) * 1e-5).astype(np.float32)
    jb = api.rates_accumulate(ctx, s["atom"], s["lam"], s["tag"], dev["temperature"], torch.from_numpy(J).cuda())
    jr = oa.jbar(ad, s["lam"], s["tag"], T.reshape(-1), J)
    assert rel(jb.cpu().numpy(), jr)[:, live].max() < 1e-10
    pops = api.se_solve(ctx, s["atom"], dev["temperature"], dev["ne"], dev["nh"], jb)
    pr = oa.se_solve(ad, T.reshape(-1), ne.reshape(-1), nh.reshape(-1), jr)
    ctx.check()
    assert rel(pops.cpu().numpy(), pr)[:, live].max() < 1e-9
    assert not pops.cpu().numpy()[:, ~live].any()


def oracle_lambda_iteration(s, n_iter, dirs, w, accelerated=False, iod=1e-2, band=None):
    ad, m, lam, tag = s["ad"], s["m"], s["lam"], s["tag"]
    T, ne, nh = m["temperature"], m["ne"], m["nh"]
    pops = oa.lte_populations(ad, T, nh)
    nz, nx = T.shape
    for _ in range(n_iter):
        eta, chi = oa.eta_chi(ad, lam, tag, T, ne, pops, m["cell_cm"])
        # the emissivity/opacity the GPU solves with are float32
        eta = eta.astype(np.float32).astype(np.float64)
        chi = chi.astype(np.float32).astype(np.float64)
        empty = omips.block_empty(eta, chi, 16)
        probes = omips.probes_of_blocks(empty, 16)
        if accelerated:
            levels, passes = omips.mip_chain(eta, chi, 3, iod, iod, 0.25, mean="linear")
            lev = omips.block_levels(passes, empty, 16, 8)
            Jp = lc.formal_solve_banded(levels, lev, 16, 8, [] if band is None else band, dirs, w, probes) \
                if band is not None else lc.formal_solve(*omips.expand(levels, lev, 8), dirs, w, probes=probes)
        else:
            Jp = lc.formal_solve(eta, chi, dirs, w, probes=probes)
        J = np.zeros((len(lam), nx * nz))
        J[:, probes] = Jp
        jb = oa.jbar(ad, lam, tag, T.reshape(-1), J)
        pops = oa.se_solve(ad, T.reshape(-1), ne.reshape(-1), nh.reshape(-1), jb).reshape((3,) + T.shape)
    return pops.reshape(3, -1)


@pytest.mark.parametrize("accelerated", [False, True])
def test_lambda_iteration_matches_oracle(setup, accelerated):
    s = setup
    api, ctx, dev, m = s["api"], s["ctx"], s["dev"], s["m"]
    dirs, w = synth.directions(16)
    n_iter = 20
    pops = api.lambda_iteration(ctx, s["atom"], s["lam"], s["tag"], dev["temperature"], dev["ne"], dev["nh"], 48, 48,
                                dirs, w, n_iter, accelerated=accelerated, iod=1.0)
    ctx.check()
    ref = oracle_lambda_iteration(s, n_iter, dirs, w, accelerated=accelerated, iod=1.0)
    live = m["temperature"].reshape(-1) > 0
    err = rel(pops.cpu().numpy(), ref)[:, live]
    assert err.max() < 1e-4, f"max population error {err.max():.3e}"


def oracle_rc_lambda_iteration(s, n_iter, C, n0, caps, accelerated, iod=1.0):
    """The same iteration with the float64 radiance-cascade oracle as formal solution."""
    from oracle import rc
    ad, m, lam, tag = s["ad"], s["m"], s["lam"], s["tag"]
    T, ne, nh = m["temperature"], m["ne"], m["nh"]
    pops = oa.lte_populations(ad, T, nh)
    nz, nx = T.shape
    dirs = synth.rc_directions(n0, C)
    for _ in range(n_iter):
        eta, chi = oa.eta_chi(ad, lam, tag, T, ne, pops, m["cell_cm"])
        eta = eta.astype(np.float32).astype(np.float64)
        chi = chi.astype(np.float32).astype(np.float64)
        empty = omips.block_empty(eta, chi, 16)
        L = eta.shape[0]
        if accelerated:
            levels, passes = omips.mip_chain(eta, chi, 3, iod, iod, 0.25, mean="linear")
            lev = omips.block_levels(passes, empty, 16, 8)
        else:
            levels, passes = [(eta, chi)], []
            lev = omips.block_levels([], empty, 16, 8, n_lambda=L)
            caps = [0] * C
        grids = [omips.expand(levels, np.where(lev >= 0, np.minimum(lev, caps[i]), -1), 8) for i in range(C)]
        J = rc.rc_solve(grids, C, n0, dirs)
        J[:, ~np.repeat(np.repeat(~empty, 16, 0), 16, 1).reshape(-1)] = 0.0
        jb = oa.jbar(ad, lam, tag, T.reshape(-1), J)
        pops = oa.se_solve(ad, T.reshape(-1), ne.reshape(-1), nh.reshape(-1), jb).reshape((3,) + T.shape)
    return pops.reshape(3, -1)


@pytest.mark.parametrize("accelerated", [False, True])
def test_cascade_lambda_iteration_matches_oracle(setup, accelerated):
    s = setup
    api, ctx, dev, m = s["api"], s["ctx"], s["dev"], s["m"]
    C, n0, caps, n_iter = 4, 4, [0, 0, 1, 2], 10
    pops = api.lambda_iteration(ctx, s["atom"], s["lam"], s["tag"], dev["temperature"], dev["ne"], dev["nh"], 48, 48,
                                None, None, n_iter, accelerated=accelerated, iod=1.0,
                                cascades={"n_cascades": C, "n0": n0, "level_cap": caps})
    ctx.check()
    ref = oracle_rc_lambda_iteration(s, n_iter, C, n0, caps, accelerated)
    live = m["temperature"].reshape(-1) > 0
    err = rel(pops.cpu().numpy(), ref)[:, live]
    assert err.max() < 1e-4, f"max population error {err.max():.3e}"
