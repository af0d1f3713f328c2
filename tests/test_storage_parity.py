"""Reduced-precision brick storage (bfloat16; float16 with per-record scales).

At MIP level 0 the records are the input S = eta/chi and chi, computed in float32 on
both sides; the oracle rounds them exactly as the format does (bfloat16: round to
nearest even of the float32 bits; float16: divide by the record's float32 maximum,
round to nearest float16, multiply back in float32), then solves in float64.  The
GPU accumulates in float32, so intensities must agree within 1e-5.  With MIP levels
the rounding acts on float32 averages the oracle forms in float64, so those runs are
compared with the float32-storage GPU result instead, within the format's resolution.
"""

import numpy as np
import pytest

import synth
from oracle import lc, mips as omips

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def f16_scaled_round(rec):
    """rec: [..., W] float32 values of one record kind."""
    m = rec.max(axis=-1, keepdims=True)
    m = np.where(m > 0, m, np.float32(1.0)).astype(np.float32)
    h = (rec / m).astype(np.float32).astype(np.float16)
    return (h.astype(np.float32) * m).astype(np.float32)


def encode(e, c):
    """Record entries (S, chi) in float32: S = eta / chi; a transparent emitter
    (chi = 0, eta > 0) is stored as S = 2^60, chi = eta 2^-60 (Eq. RteIntegral's
    limit chi -> 0 of S (1 - e^{-chi ds}) = eta ds)."""
    pos = c > 0
    S = np.zeros_like(e)
    S[pos] = e[pos] / c[pos]
    em = (~pos) & (e > 0)
    S[em] = np.float32(2.0 ** 60)
    x = c.copy()
    x[em] = e[em] * np.float32(2.0 ** -60)
    return S.astype(np.float32), x.astype(np.float32)


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(np.abs(b), 1e-30)


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


def gpu_line(ctx, m):
    from paper_2511_08498_gb300 import api
    t = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda()
         for k in ("chi_c", "s_c", "s_l", "ratio", "dld", "dlam")}
    return api.synth_static_line(ctx, t["chi_c"], t["s_c"], t["s_l"], t["ratio"], t["dld"], t["dlam"])


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("W", [4, 8])
def test_level0_storage_matches_emulated_oracle(ctx, storage, W):
    from paper_2511_08498_gb300 import api
    nx, nz, L = 96, 80, 16
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=synth.SEED_BASE + 800)
    eg, cg = gpu_line(ctx, m)
    dirs, w = synth.directions(12)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    mp = api.mips_build(ctx, grid, eg, cg, W, 0, 1.0, 1.0, 0.25, storage=storage)
    J, I, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w, want_intensity=True)
    ctx.check()
    # the GPU's float32 eta/chi (the method's input here) -> records -> rounding
    e32 = eg.cpu().numpy().reshape(L, nz, nx)
    c32 = cg.cpu().numpy().reshape(L, nz, nx)
    S32, c32 = encode(e32, c32)
    if storage == 1:
        Sr, cr = bf16_round(S32), bf16_round(c32)
    else:
        rec = lambda a: np.moveaxis(a.reshape(L // W, W, nz, nx), 1, -1)
        unrec = lambda a: np.moveaxis(a, -1, 1).reshape(L, nz, nx)
        Sr, cr = unrec(f16_scaled_round(rec(S32))), unrec(f16_scaled_round(rec(c32)))
    er = Sr.astype(np.float64) * cr.astype(np.float64)
    empty = omips.block_empty(e32, c32, 16)
    probes = omips.probes_of_blocks(empty, 16)
    Jr, Ir = lc.formal_solve(er, cr.astype(np.float64), dirs, w, probes=probes, want_intensity=True)
    assert rel(I.cpu().numpy()[:, :, probes], Ir).max() < 1e-5
    assert rel(J.cpu().numpy()[:, probes], Jr).max() < 1e-5


@pytest.mark.parametrize("storage,bound", [(1, 2e-2), (2, 2e-3)])
def test_mip_storage_close_to_float32(ctx, storage, bound):
    from paper_2511_08498_gb300 import api
    nx, nz, L = 128, 96, 16
    m = synth.sparse_line_atmosphere(nx, nz, n_lambda=L, seed=synth.SEED_BASE + 810)
    eg, cg = gpu_line(ctx, m)
    dirs, w = synth.directions(16)
    grid = api.grid_build(ctx, nx, nz, eg, cg)
    ref = api.mips_build(ctx, grid, eg, cg, 8, 3, 1.0, 1.0, 0.25)
    Jf, _, _ = api.formal_solve_hdda(ctx, grid, ref, dirs, w, band=[6, 24, 96])
    mp = api.mips_build(ctx, grid, eg, cg, 8, 3, 1.0, 1.0, 0.25, storage=storage)
    Jr, _, _ = api.formal_solve_hdda(ctx, grid, mp, dirs, w, band=[6, 24, 96])
    ctx.check()
    # identical level maps (decided before rounding), so only the stored values differ
    assert torch.equal(mp.words, ref.words)
    probes = torch.from_numpy(omips.probes_of_blocks(
        np.asarray(api.unpack_states(ref.words.cpu().numpy(), grid.n_blocks)[0] < 0).reshape(grid.nbz, grid.nbx),
        16)).long().cuda()
    e = rel(Jr[:, probes].cpu().numpy(), Jf[:, probes].cpu().numpy().astype(np.float64))
    assert e.max() < bound, e.max()


# Measured on the 48 x 48 populations atmosphere below (20 Lambda steps):
#   float16 + per-record scales: max below 1e-3, inside the paper's 0.5 % bar;
#   bfloat16: max 2.4 %, p99 0.55 % -- its 8-bit significand misses the bar, so
#   the bound here only guards against regressions and the format is reported,
#   not recommended, for the population workload.
@pytest.mark.parametrize("storage,bound,p99", [(1, 5e-2, 1e-2), (2, 5e-3, 1e-3)])
def test_lambda_iteration_populations_with_reduced_storage(ctx, storage, bound, p99):
    """Populations after a 20-step Lambda iteration whose bricks are stored in the
    reduced format, against the same iteration with float32 bricks.  The records
    carry 8 (bfloat16) or 11 (float16) significant bits; the error they leave in
    the populations is what decides whether the format is usable for the method."""
    from paper_2511_08498_gb300 import api
    from synth.atom import line_wavelength_grid, populations_atmosphere, three_level_atom
    ad = three_level_atom()
    m = populations_atmosphere(48, 48, seed=synth.SEED_BASE + 500)
    lam, tag = line_wavelength_grid(8, 4)
    atom = api.Atom.from_dict(ad, m["cell_cm"])
    dev = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in ("temperature", "ne", "nh")}
    dirs, w = synth.directions(16)
    run = lambda st: api.lambda_iteration(ctx, atom, lam, tag, dev["temperature"], dev["ne"], dev["nh"], 48, 48,
                                          dirs, w, 20, accelerated=True, iod=1.0, storage=st).cpu().numpy()
    ref, red = run(0), run(storage)
    ctx.check()
    live = m["temperature"].reshape(-1) > 0
    err = rel(red, ref)[:, live]
    print(f"storage {storage}: population error max {err.max():.3e} p99 {np.quantile(err, 0.99):.3e}")
    assert err.max() < bound
    assert np.quantile(err, 0.99) < p99
