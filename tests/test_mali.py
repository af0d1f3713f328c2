"""MALI on the GPU (dex_mali_rates, dex_se_solve_preconditioned,
dex_max_rel_change; api.mali_iteration) vs the float64 MALI oracle.

Tolerances, from the arithmetic:
* preconditioned rates from the same populations: the kernel gets the oracle's
  own-cell-free J (J minus Lambda* S in float64, rounded to float32) and works
  in float64 except the own-cell escape sum_d w_d e^{-chi l_d}, taken in float32
  (relative error ~1e-7); rho = 1 - Psibar is evaluated without cancellation
  (the oracle's float64 1 - Psibar loses up to ~1e-16 / rho relative): rho
  within 1e-6 relative; Jbar_eff within 1e-7 of the line's Jbar scale (the
  float32 rounding of the own-cell-free J);
* SE with the same preconditioned rates: float64 elimination on both sides, 1e-9;
* the whole iteration (the GPU's formal solution is float32, 1e-5 of the
  oracle's, and MALI carries that into every update): after a fixed number of
  updates the populations within 1e-3 relative, the convergence history within
  2% relative of the oracle's, and the converged run needs the same number of
  updates as the oracle's +-1.
"""

import numpy as np
import pytest

import synth
from oracle import atom as oa, lc, mali, mips as omips
from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NDIR = 48, 16


@pytest.fixture(scope="module")
def case():
    from paper_2511_08498_gb300 import api
    ctx = api.Context(0)
    ad = three_level_atom()
    m = populations_atmosphere(N, N, seed=synth.SEED_BASE + 4)
    lam, tag = line_wavelength_grid(t_ref=1e5)
    dirs, w = synth.directions(NDIR)
    dev = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in ("temperature", "ne", "nh")}
    host = {k: m[k].astype(np.float64).reshape(-1) for k in ("temperature", "ne", "nh")}
    atom = api.Atom.from_dict(ad, m["cell_cm"])
    return dict(api=api, ctx=ctx, ad=ad, m=m, lam=lam, tag=tag, dirs=dirs, w=w, dev=dev, host=host, atom=atom)


def oracle_solve_J(c):
    lam, dirs, w = c["lam"], c["dirs"], c["w"]

    def solve_J(eta, chi):
        e, x = eta.reshape(-1, N, N), chi.reshape(-1, N, N)
        probes = omips.probes_of_blocks(omips.block_empty(e, x, 16), 16)
        J = np.zeros((lam.size, N * N))
        J[:, probes] = lc.formal_solve(e, x, dirs, w, probes=probes)
        return J
    return solve_J


def test_rates_and_se_match_oracle(case):
    c = case
    api, ctx, ad, h, lam, tag = c["api"], c["ctx"], c["ad"], c["host"], c["lam"], c["tag"]
    T, ne, nh = h["temperature"], h["ne"], h["nh"]
    # populations away from LTE, the oracle's J for them and its own-cell-free part
    pops = oa.lte_populations(ad, T, nh) * np.array([[1.2], [0.8], [0.6]])
    eta, chi = oa.eta_chi(ad, lam, tag, T, ne, pops, c["m"]["cell_cm"])
    J64 = oracle_solve_J(c)(eta, chi)
    with np.errstate(invalid="ignore", divide="ignore"):
        S = np.where(chi > 0, eta / np.where(chi > 0, chi, 1.0), 0.0)
    Jext = (J64 - mali.lambda_star(chi, c["dirs"], c["w"]) * S).astype(np.float32)
    J = J64.astype(np.float32)
    Jg = torch.from_numpy(Jext).cuda()
    pg = torch.from_numpy(pops).cuda()
    rho, jeff = api.mali_rates(ctx, c["atom"], lam, tag, c["dev"]["temperature"], c["dev"]["ne"], pg, Jg, c["dirs"],
                               c["w"])
    ctx.check()
    # the oracle from the same float32 J
    eta_l, chi_l = mali.line_eta_chi(ad, lam, tag, T, pops, c["m"]["cell_cm"])
    lstar = mali.lambda_star(chi, c["dirs"], c["w"])
    psibar, jeff_r = mali.preconditioned(ad, lam, tag, T, J64, chi, eta_l, chi_l, lstar)
    live = T > 0
    rho_r = 1.0 - psibar
    r = rho.cpu().numpy()
    assert np.all(r[:, ~live] == 0)
    np.testing.assert_allclose(r[:, live], rho_r[:, live], rtol=1e-6, atol=1e-15)
    scale = np.abs(oa.jbar(ad, lam, tag, T, J.astype(np.float64))).max(axis=1, keepdims=True)
    assert np.abs(jeff.cpu().numpy()[:, live] - jeff_r[:, live]).max() <= 1e-7 * scale.max()
    # SE with the preconditioned rates: GPU rates into both solves
    new = api.se_solve_preconditioned(ctx, c["atom"], c["dev"]["temperature"], c["dev"]["ne"], c["dev"]["nh"], rho,
                                      jeff)
    ctx.check()
    P = mali.rate_matrix(ad, T, ne, 1.0 - rho.cpu().numpy(), jeff.cpu().numpy())
    ref = mali.solve_populations(P, nh, live)
    np.testing.assert_allclose(new.cpu().numpy()[:, live], ref[:, live], rtol=1e-9)
    # convergence measure
    out = api.max_rel_change(ctx, c["dev"]["temperature"], pg, new)
    ctx.check()
    want = np.max(np.abs(ref[:, live] - pops[:, live]) / ref[:, live])
    assert abs(out.item() - want) <= 1e-9 * want


def test_iteration_matches_oracle(case):
    c = case
    api, ctx, ad, h = c["api"], c["ctx"], c["ad"], c["host"]
    K = 12
    pg, n, hist = api.mali_iteration(ctx, c["atom"], c["lam"], c["tag"], c["dev"]["temperature"], c["dev"]["ne"],
                                     c["dev"]["nh"], N, N, c["dirs"], c["w"], n_iter=K)
    ctx.check()
    pr, nr, hr = mali.iterate(ad, c["lam"], c["tag"], h["temperature"], h["ne"], h["nh"], c["m"]["cell_cm"],
                              oracle_solve_J(c), c["dirs"], c["w"], tol=0.0, max_iter=K)
    live = h["temperature"] > 0
    e = np.abs(pg.cpu().numpy()[:, live] / pr[:, live] - 1)
    assert e.max() < 1e-3, e.max()
    np.testing.assert_allclose(hist, hr, rtol=2e-2)


def test_converged_iteration_count_matches_oracle(case):
    c = case
    api, ctx, ad, h = c["api"], c["ctx"], c["ad"], c["host"]
    pg, n, hist = api.mali_iteration(ctx, c["atom"], c["lam"], c["tag"], c["dev"]["temperature"], c["dev"]["ne"],
                                     c["dev"]["nh"], N, N, c["dirs"], c["w"], tol=1e-3, max_iter=150)
    ctx.check()
    pr, nr, hr = mali.iterate(ad, c["lam"], c["tag"], h["temperature"], h["ne"], h["nh"], c["m"]["cell_cm"],
                              oracle_solve_J(c), c["dirs"], c["w"], tol=1e-3, max_iter=150)
    assert hist[-1] < 1e-3 and hr[-1] < 1e-3
    assert abs(n - nr) <= 1, (n, nr)
    live = h["temperature"] > 0
    assert np.abs(pg.cpu().numpy()[:, live] / pr[:, live] - 1).max() < 1e-3


def test_accelerated_iteration_converges_near_plain(case):
    """MALI with the accelerated formal solution (VLM 0-3, IoD 1, distance limits)
    converges too, to populations within the method's error of the plain ones."""
    c = case
    api, ctx = c["api"], c["ctx"]
    args = (ctx, c["atom"], c["lam"], c["tag"], c["dev"]["temperature"], c["dev"]["ne"], c["dev"]["nh"], N, N,
            c["dirs"], c["w"])
    pp, n_p, _ = api.mali_iteration(*args, tol=1e-3, max_iter=150)
    pa, n_a, ha = api.mali_iteration(*args, tol=1e-3, max_iter=150, accelerated=True, iod=1.0,
                                     band=[6.0, 24.0, 96.0])
    ctx.check()
    live = c["host"]["temperature"] > 0
    assert ha[-1] < 1e-3 and n_a < 150
    err = np.abs(pa.cpu().numpy()[:, live] / pp.cpu().numpy()[:, live] - 1)
    assert np.percentile(err, 99.9) < 5e-3


@pytest.mark.parametrize("accelerated", [False, True])
def test_own_cell_emission_left_out(case, accelerated):
    """dex_ctx_set_own_cell(ctx, 0): the solves return J minus the own cell's
    Lambda* S (the oracle's float64 J and Lambda* S, subtracted): within 1e-5 of
    J everywhere and 1e-5 relative wherever the remainder is at least 1e-4 of J."""
    c = case
    api, ctx, ad, h, lam, tag = c["api"], c["ctx"], c["ad"], c["host"], c["lam"], c["tag"]
    T, ne, nh = h["temperature"], h["ne"], h["nh"]
    pops = oa.lte_populations(ad, T, nh)
    eta, chi = oa.eta_chi(ad, lam, tag, T, ne, pops, c["m"]["cell_cm"])
    eg = torch.from_numpy(eta.astype(np.float32)).cuda()
    cg = torch.from_numpy(chi.astype(np.float32)).cuda()
    grid = api.grid_build(ctx, N, N, eg, cg)
    ctx.set_own_cell(False)
    try:
        if accelerated:
            mp = api.mips_build(ctx, grid, eg, cg, 8, 3, 1e30, 1e30, 0.25)
            J, _, _ = api.formal_solve_hdda(ctx, grid, mp, c["dirs"], c["w"], band=[6.0, 24.0, 96.0])
        else:
            planes = api.pack_planes(ctx, eg, cg, 8)
            J, _, _ = api.formal_solve_dense(ctx, N, N, lam.size, 8, planes, c["dirs"], c["w"])
        ctx.check()
    finally:
        ctx.set_own_cell(True)
    e32, c32 = eta.astype(np.float32).astype(np.float64), chi.astype(np.float32).astype(np.float64)
    probes = omips.probes_of_blocks(omips.block_empty(e32.reshape(-1, N, N), c32.reshape(-1, N, N), 16), 16)
    if accelerated:
        levels, passes = omips.mip_chain(e32.reshape(-1, N, N), c32.reshape(-1, N, N), 3, 1e30, 1e30, 0.25,
                                         mean="linear")
        lev = omips.block_levels(passes, omips.block_empty(e32.reshape(-1, N, N), c32.reshape(-1, N, N), 16), 16, 8)
        Jr = lc.formal_solve_banded(levels, lev, 16, 8, [6.0, 24.0, 96.0], c["dirs"], c["w"], probes)
    else:
        Jr = lc.formal_solve(e32.reshape(-1, N, N), c32.reshape(-1, N, N), c["dirs"], c["w"], probes=probes)
    with np.errstate(invalid="ignore", divide="ignore"):
        S = np.where(c32 > 0, e32 / np.where(c32 > 0, c32, 1.0), 0.0)
    own = (mali.lambda_star(c32, c["dirs"], c["w"]) * S)[:, probes]
    ext = Jr - own
    got = J.cpu().numpy()[:, probes].astype(np.float64)
    assert np.abs(got - ext).max() <= 1e-5 * np.abs(Jr).max()
    big = ext > 1e-4 * Jr
    assert big.mean() > 0.1
    assert (np.abs(got - ext)[big] / ext[big]).max() < 1e-5
    # other solvers refuse the setting
    ctx.set_own_cell(False)
    with pytest.raises(api.DexError):
        api.formal_solve_hdda(ctx, grid, api.mips_build(ctx, grid, eg, cg, 4, 3, 1.0, 1.0, 0.25), c["dirs"], c["w"])
    ctx.set_own_cell(True)
