"""Velocity interpolation (Section 3.1) on the GPU vs the float64 oracle.

The grid values come from the float32 Voigt function, within 2.5e-5 relative of
the oracle's float64 HUM1WEI24 (test_cav_parity derives the bound and the 1e-4
tolerance it implies for intensities); interpolation and traversal add only
float32 rounding, so intensities are compared at 1e-4.  Block levels
(rest-frame IoD) must agree exactly.
"""

import numpy as np
import pytest

import synth
from oracle import mips as omips, velinterp as ov
from oracle.cav import param_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(np.abs(b), 1e-30)


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_08498_gb300 import api
    return api.Context(0)


@pytest.mark.parametrize("max_mip,iod,band,cm,test_dirs", [(0, 1.0, None, 0.25, 0), (2, 1.0, None, 0.25, 0),
                                                            (3, 1e9, [5.3, 21.7, 40.2], 0.25, 0),
                                                            (3, 100.0, [5.3, 21.7, 40.2], 0.0, 8)])
def test_velinterp_matches_oracle(ctx, max_mip, iod, band, cm, test_dirs):
    from paper_2511_08498_gb300 import api
    from levels_util import robust_level_mask_multi
    m = synth.dynamic_line_atmosphere(128, 96, n_lambda=16, seed=synth.SEED_BASE + 700)
    dirs, w = synth.directions(8)
    f = {k: torch.from_numpy(np.ascontiguousarray(m[k]).reshape(-1)).cuda() for k in api.CAV_FIELDS}
    grid = api.cav_grid_build(ctx, 128, 96, f)
    mp = api.vel_mips_build(ctx, grid, f, m["dv"], m["c_kms"], 8, max_mip, iod, iod, cm, test_dirs=test_dirs)
    J, I, _ = api.formal_solve_velinterp(ctx, grid, mp, dirs, w, band=band, want_intensity=True)
    ctx.check()
    P0 = param_arrays(m)
    empty = omips.block_empty(np.stack([m["eta_star"], m["eta_c"]]), np.stack([m["chi_star"], m["chi_c"]]), 16)
    if max_mip > 0:
        lev, st = ov.levels(P0, m["dv"], m["c_kms"], empty, 16, 8, max_mip, iod, cm, stats=True,
                            n_test_dirs=test_dirs)
    else:
        lev = omips.block_levels([], empty, 16, 8, n_lambda=16)
    if test_dirs:   # the directional tests change levels here, and no decision sits on a threshold
        assert robust_level_mask_multi(st, lev, 8, 16, max_mip, iod, iod, cm).all()
        assert (ov.levels(P0, m["dv"], m["c_kms"], empty, 16, 8, max_mip, iod, cm) != lev).any()
    nbz, nbx = empty.shape
    np.testing.assert_array_equal(api.unpack_states(mp.words.cpu().numpy(), nbz * nbx).reshape(lev.shape), lev)
    grids = ov.velocity_grids(P0, m["dv"], m["c_kms"], max_mip)
    probes = omips.probes_of_blocks(empty, 16)
    Jr, Ir = ov.formal_solve(grids, lev, 16, 8, dirs, w, probes, band=band, want_intensity=True)
    assert rel(I.cpu().numpy()[:, :, probes], Ir).max() < 1e-4
    assert rel(J.cpu().numpy()[:, probes], Jr).max() < 1e-4
