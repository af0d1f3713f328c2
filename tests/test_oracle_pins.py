"""Pins of the float64 oracle against facts that do not come from the oracle itself:
exact rational ray/grid geometry, closed-form solutions of the transfer equation,
brute-force fine sub-stepping, a hand-computed two-voxel case, and numbers the
paper prints (MIP storage factors, block-state packing).
"""

import math
from fractions import Fraction as F

import numpy as np
import pytest

import synth
from oracle import lc, lines, mips


# ---------------------------------------------------------------- geometry ----

def exact_cells(nx, nz, o, d):
    """Cell-by-cell walk in exact rational arithmetic (different algorithm from the
    oracle's sorted plane crossings).  Returns [(cell, length_in_t)]."""
    ox, oz = F(o[0]), F(o[1])
    dx, dz = F(d[0]), F(d[1])

    def exit_t(oc, dc, n):
        if dc > 0:
            return (n - oc) / dc
        if dc < 0:
            return (0 - oc) / dc
        return None

    cands = [t for t in (exit_t(ox, dx, nx), exit_t(oz, dz, nz)) if t is not None]
    tex = min(cands)
    i, j = math.floor(ox), math.floor(oz)
    t = F(0)
    out = []
    while t < tex:
        tx = ((i + 1 - ox) / dx if dx > 0 else (i - ox) / dx) if dx != 0 else None
        tz = ((j + 1 - oz) / dz if dz > 0 else (j - oz) / dz) if dz != 0 else None
        nxt = min(v for v in (tx, tz, tex) if v is not None)
        if nxt > t:
            out.append((j * nx + i, nxt - t))
        if nxt == tex:
            break
        if tx is not None and tx == nxt:
            i += 1 if dx > 0 else -1
        if tz is not None and tz == nxt:
            j += 1 if dz > 0 else -1
        t = nxt
    return out, tex


GEOM_CASES = [
    (7, 5, (F(1, 2), F(1, 2)), (1, 1)),          # passes exactly through corners
    (7, 5, (F(7, 2), F(5, 2)), (-1, 1)),
    (6, 6, (F(5, 2), F(3, 2)), (F(3, 5), F(4, 5))),
    (6, 6, (F(5, 2), F(7, 2)), (F(-5, 13), F(-12, 13))),
    (9, 4, (F(3, 2), F(1, 2)), (1, 0)),          # axis parallel
    (9, 4, (F(3, 2), F(7, 2)), (0, -1)),
    (8, 8, (F(1, 2), F(13, 2)), (F(8, 17), F(-15, 17))),
    (5, 9, (F(9, 2), F(1, 2)), (-2, 3)),
]


@pytest.mark.parametrize("nx,nz,o,d", GEOM_CASES)
def test_segments_match_exact_rational_walk(nx, nz, o, d):
    exact, tex = exact_cells(nx, nz, o, d)
    cells, lens = lc.ray_segments(nx, nz, (float(o[0]), float(o[1])), (float(d[0]), float(d[1])))
    assert [c for c, _ in exact] == list(cells)
    np.testing.assert_allclose(lens, [float(L) for _, L in exact], rtol=0, atol=1e-12)
    assert abs(lens.sum() - float(tex)) < 1e-12


def test_segment_lengths_sum_to_exit_distance():
    dirs, _ = synth.directions(16)
    nx, nz = 13, 11
    for (i, j) in [(0, 0), (6, 5), (12, 10), (3, 9)]:
        o = (i + 0.5, j + 0.5)
        for d in dirs.astype(np.float64):
            _, lens = lc.ray_segments(nx, nz, o, d)
            tx = (nx - o[0]) / d[0] if d[0] > 0 else (-o[0] / d[0] if d[0] < 0 else np.inf)
            tz = (nz - o[1]) / d[1] if d[1] > 0 else (-o[1] / d[1] if d[1] < 0 else np.inf)
            assert abs(lens.sum() - min(tx, tz)) < 1e-10


def test_dense_segment_count_small_closed_form():
    # Axis-parallel rays on an n x n grid from every cell centre: a ray toward +x
    # from column i crosses n - i cells, so the total over 4 directions is
    # 4 * n * sum_{i}(n - i) = 2 n^2 (n + 1).
    n = 9
    dirs, _ = synth.directions(4, offset=0.0)
    probes = np.arange(n * n, dtype=np.int32)
    assert lc.count_segments(n, n, dirs, probes) == 2 * n * n * (n + 1)


# ------------------------------------------------------- closed-form RTE ----

def _texit(nx, nz, o, d):
    tx = (nx - o[0]) / d[0] if d[0] > 0 else (-o[0] / d[0] if d[0] < 0 else np.inf)
    tz = (nz - o[1]) / d[1] if d[1] > 0 else (-o[1] / d[1] if d[1] < 0 else np.inf)
    return min(tx, tz)


def test_uniform_slab_closed_form():
    nx, nz = 12, 9
    chi0, S = 0.37, 2.5
    eta = np.full((1, nz, nx), chi0 * S)
    chi = np.full((1, nz, nx), chi0)
    dirs, w = synth.directions(8)
    d64 = dirs.astype(np.float64)
    for ibc in (0.0, 1.7):
        J, I = lc.formal_solve(eta, chi, d64, w, i_bc=ibc, want_intensity=True)
        for p in [0, 17, nx * nz - 1, 50]:
            o = (p % nx + 0.5, p // nx + 0.5)
            for k in range(8):
                tau = chi0 * _texit(nx, nz, o, d64[k])
                ref = S * (1 - math.exp(-tau)) + ibc * math.exp(-tau)
                assert abs(I[0, k, p] - ref) <= 1e-13 * max(1.0, abs(ref))
            assert abs(J[0, p] - np.dot(w, I[0, :, p])) < 1e-13


def test_transparent_and_pure_emission():
    nx, nz = 10, 7
    dirs, w = synth.directions(12)
    d64 = dirs.astype(np.float64)
    zero = np.zeros((1, nz, nx))
    J = lc.formal_solve(zero, zero, d64, w, i_bc=3.25)
    np.testing.assert_array_equal(J, 3.25 * np.asarray(w, np.float64).sum())
    eta = np.full((1, nz, nx), 0.6)
    J, I = lc.formal_solve(eta, zero, d64, w, i_bc=1.0, want_intensity=True)
    for p in [0, 33, nx * nz - 1]:
        o = (p % nx + 0.5, p // nx + 0.5)
        for k in range(12):
            assert abs(I[0, k, p] - (1.0 + 0.6 * _texit(nx, nz, o, d64[k]))) < 1e-12


def test_exponential_atmosphere_row_sums():
    # chi depends on z only, taken as the exact cell average of chi0 exp(-z/H);
    # S constant.  For an upward ray from row j0, the optical depth is
    # (0.5 chi_j0 + sum_{j > j0} chi_j) / sin(theta), independent of how the
    # x planes cut the path.
    nx, nz, H, chi0, S = 100, 24, 6.0, 0.8, 1.3
    j = np.arange(nz)
    chi_row = chi0 * H * (np.exp(-j / H) - np.exp(-(j + 1) / H))
    chi = np.broadcast_to(chi_row[:, None], (nz, nx)).copy()[None]
    eta = S * chi
    th = np.array([0.9, 1.2, 1.5707963267948966, 2.3])
    dirs = np.stack([np.cos(th), np.sin(th)], 1)
    w = np.ones(len(th))
    for j0 in (0, 5, 11):
        probes = np.array([j0 * nx + 50], dtype=np.int32)  # every ray exits the top
        _, I = lc.formal_solve(eta, chi, dirs, w, probes=probes, want_intensity=True)
        for k, t in enumerate(th):
            tau = (0.5 * chi_row[j0] + chi_row[j0 + 1:].sum()) / math.sin(t)
            ref = S * (1 - math.exp(-tau))
            assert abs(I[0, k, 0] - ref) < 1e-12 * ref
        # and the continuous optical depth of exp(-z/H) from z0 = j0 + 1 up to nz
        # plus the half cell is recovered for the vertical ray
        tau_cont = (chi0 * H * (math.exp(-(j0 + 1) / H) - math.exp(-nz / H)) + 0.5 * chi_row[j0])
        assert abs(I[0, 2, 0] - S * (1 - math.exp(-tau_cont))) < 1e-12


def test_two_voxel_upwind_by_hand():
    # Ray from the centre of voxel A (0.5, 0.5) toward +x through voxel B to the
    # boundary x = 2.  Radiation reaching A comes from B first (upwind), then
    # crosses half of A:  I = [S_B (1 - e^{-tau_B})] e^{-tau_A} + S_A (1 - e^{-tau_A}),
    # tau_B = 0.9 * 1, tau_A = 0.2 * 0.5; S_B = 3, S_A = 0.5.
    eta = np.array([[[0.5 * 0.2, 3.0 * 0.9]]])
    chi = np.array([[[0.2, 0.9]]])
    _, I = lc.formal_solve(eta, chi, [[1.0, 0.0]], [1.0], probes=np.array([0], np.int32), want_intensity=True)
    # hand value: 3*(1-exp(-0.9)) = 1.78029102..., times exp(-0.1) = 1.61087393...;
    # plus 0.5*(1-exp(-0.1)) = 0.04758129...
    assert abs(I[0, 0, 0] - 1.6584552216) < 2e-10
    # the opposite ordering (downwind) would give 0.5*(1-e^-0.1)*e^-0.9 + 1.7803 = 1.79964...
    assert abs(I[0, 0, 0] - 1.79964) > 0.1


def _substep_intensity(eta, chi, o, d, ibc, h):
    """Brute-force: march from the exit point back to the origin in steps of h,
    looking the voxel up at each sub-step midpoint, exact update per sub-step."""
    nz, nx = eta.shape
    tex = _texit(nx, nz, o, d)
    n = int(math.ceil(tex / h))
    I = ibc
    for s in range(n - 1, -1, -1):
        t0, t1 = s * h, min((s + 1) * h, tex)
        tm = 0.5 * (t0 + t1)
        i = min(max(int(math.floor(o[0] + tm * d[0])), 0), nx - 1)
        j = min(max(int(math.floor(o[1] + tm * d[1])), 0), nz - 1)
        x, e, L = chi[j, i], eta[j, i], t1 - t0
        if x > 0:
            I = I * math.exp(-x * L) + e / x * (1 - math.exp(-x * L))
        else:
            I = I + e * L
    return I


def test_brute_force_substepping():
    rng = np.random.default_rng(7)
    nx, nz = 6, 5
    chi = rng.uniform(0.0, 2.0, (nz, nx))
    chi[1, 2] = 0.0
    S = rng.uniform(0.5, 3.0, (nz, nx))
    eta = chi * S
    eta[1, 2] = 0.4  # a pure emitter
    th = [0.3, 1.9, 3.5, 4.4, 5.9]
    dirs = np.array([[math.cos(t), math.sin(t)] for t in th])
    _, I = lc.formal_solve(eta[None], chi[None], dirs, np.ones(len(th)), i_bc=0.25, want_intensity=True)
    for p in [0, 13, 29]:
        o = (p % nx + 0.5, p // nx + 0.5)
        for k in range(len(th)):
            ref = _substep_intensity(eta, chi, o, dirs[k], 0.25, 2e-4)
            assert abs(I[0, k, p] - ref) < 3e-3 * max(ref, 1e-3)


# ------------------------------------------------------------- line model ----

def test_line_synthesis_closed_forms():
    chi_c = np.array([[1.0, 0.0], [2.0, 1e-3]])
    s_c = np.array([[1.5, 0.0], [0.7, 2.0]])
    s_l = np.array([[0.5, 0.0], [0.2, 1.0]])
    ratio = np.array([[100.0, 100.0], [1e5, 10.0]])
    dld = np.array([[1.0, 2.0], [3.0, 1.5]])
    dlam = np.array([0.0, 1.0, 40.0])
    eta, chi = lines.line_eta_chi(chi_c, s_c, s_l, ratio, dld, dlam)
    # line centre: chi = chi_c (1 + ratio)
    np.testing.assert_allclose(chi[0], chi_c * (1 + ratio), rtol=1e-15)
    np.testing.assert_allclose(eta[0], chi_c * s_c + ratio * chi_c * s_l, rtol=1e-15)
    # one Doppler width from centre of the dld = 1 cell: factor e^-1
    assert abs(chi[1, 0, 0] - (1.0 + 100.0 * math.exp(-1.0))) < 1e-12
    # far wing: continuum only
    np.testing.assert_allclose(chi[2], chi_c, rtol=1e-12)
    np.testing.assert_allclose(eta[2], chi_c * s_c, rtol=1e-12)
    assert chi[:, 0, 1].max() == 0 and eta[:, 0, 1].max() == 0


# ----------------------------------------------- MIP chain and block map ----

def test_mip_chain_storage_factors_printed_in_paper():
    # Section 2.1: the full MIP chain costs 1.33x MIP 0 in 2D and 1.14x in 3D.
    f2 = sum(4.0 ** -m for m in range(0, 30))
    f3 = sum(8.0 ** -m for m in range(0, 30))
    assert round(f2, 2) == 1.33 and round(f3, 2) == 1.14
    # and the chain the oracle builds for a 64^2 grid has exactly sum 4^-m x MIP 0
    e = np.ones((1, 64, 64))
    levels, _ = mips.mip_chain(e, e, 6, 1.0, 1.0)
    sizes = [lv[0].size for lv in levels]
    assert sum(sizes) / sizes[0] == sum(4.0 ** -m for m in range(7))
    # Section 2.2: MIP 0 and 1 hold 94% of the 2D storage
    assert round((1 + 0.25) / (4.0 / 3.0), 2) == 0.94


def test_block_state_packing_printed_in_paper():
    # Section 2.3.1: 6 states in 3 bits -> 21 blocks per 64-bit word; a 512^2 model
    # with 16^2 blocks needs 49 words (392 B).
    lev = np.zeros((32, 32), dtype=np.int32)
    words = mips.pack_states(lev)
    assert words.size == 49 and words.nbytes == 392
    rng = np.random.default_rng(3)
    lev = rng.integers(-1, 5, size=(32, 32))
    words = mips.pack_states(lev)
    np.testing.assert_array_equal(mips.unpack_states(words, 1024), lev.reshape(-1))
    # block 0 in the low 3 bits, block 20 in bits 60..62, block 21 starts word 1
    w = mips.pack_states(np.array([[4] + [-1] * 19 + [0, 2]]))
    assert int(w[0]) & 7 == 5 and (int(w[0]) >> 60) & 7 == 1 and int(w[1]) & 7 == 3


def test_morton_layout_by_hand():
    empty = np.zeros((4, 4), dtype=bool)
    active, offset = mips.block_layout(empty)
    # Z-order over (bx, bz): (0,0) (1,0) (0,1) (1,1) (2,0) (3,0) (2,1) (3,1) (0,2) ...
    assert list(active) == [0, 1, 4, 5, 2, 3, 6, 7, 8, 9, 12, 13, 10, 11, 14, 15]
    empty[0, 1] = empty[2, 2] = True
    active, offset = mips.block_layout(empty)
    assert list(active) == [0, 4, 5, 2, 3, 6, 7, 8, 9, 12, 13, 11, 14, 15]
    assert offset[0, 1] == -1 and offset[2, 2] == -1 and offset[1, 0] == 1


def test_iod_by_hand():
    # One 2x2 group at level 1 (Ds = 2), children chi = (1, 2, 4, 8), eta = chi:
    # X = ln(2 chi) = ln2 * (1, 2, 3, 4): mean 2.5 ln2 = 1.732868, population
    # variance 1.25 ln2^2 = 0.600561, IoD = 0.5 ln2 = 0.346574.
    chi = np.array([[[1.0, 2.0], [4.0, 8.0]]])
    _, passes = mips.mip_chain(chi, chi, 1, 0.35, 0.35, chi_ds_min=0.0)
    assert passes[0].all()
    _, passes = mips.mip_chain(chi, chi, 1, 0.34, 0.34, chi_ds_min=0.0)
    assert not passes[0].any()
    # always-average rule: max child chi * Ds = 16 < 17 -> passes whatever the IoD
    _, passes = mips.mip_chain(chi, chi, 1, 0.0, 0.0, chi_ds_min=17.0)
    assert passes[0].all()
    # the stored value: geometric mean (1*2*4*8)^(1/4) = 2^1.5 in log mode, 3.75 linear
    levels, _ = mips.mip_chain(chi, chi, 1, 1.0, 1.0)
    assert abs(levels[1][1][0, 0, 0] - 2.0 ** 1.5) < 1e-14
    levels, _ = mips.mip_chain(chi, chi, 1, 1.0, 1.0, mean="linear")
    assert levels[1][1][0, 0, 0] == 3.75


def test_mixed_zero_group_needs_always_average_rule():
    chi = np.array([[[0.0, 0.1], [0.1, 0.1]]])
    levels, passes = mips.mip_chain(chi, chi, 1, 1e9, 1e9, chi_ds_min=0.0)
    assert not passes[0].any()
    levels, passes = mips.mip_chain(chi, chi, 1, 1e9, 1e9, chi_ds_min=0.25)  # 0.1 * 2 < 0.25
    assert passes[0].all() and abs(levels[1][1][0, 0, 0] - 0.075) < 1e-15


def test_homogeneous_blocks_reach_max_level_and_match_plain():
    # Section 1.1: for homogeneous parameters the averaged formulation equals the
    # true one, so the accelerated solution equals the plain one.
    nx = nz = 32
    eta = np.full((2, nz, nx), 1.1)
    chi = np.full((2, nz, nx), 0.7)
    levels, passes = mips.mip_chain(eta, chi, 3, 1e-3, 1e-3)
    empty = mips.block_empty(eta, chi, 16)
    lev = mips.block_levels(passes, empty, 16, 8)
    assert (lev == 3).all()
    e2, c2 = mips.expand(levels, lev, 8)
    np.testing.assert_allclose(e2, eta, rtol=1e-15)
    np.testing.assert_allclose(c2, chi, rtol=1e-15)


def test_block_level_is_minimum_over_wavelength_batch():
    nx = nz = 16
    eta = np.full((3, nz, nx), 1.0)
    chi = np.full((3, nz, nx), 2.0)
    chi[1, 5, 9] = 200.0      # a spike at wavelength 1 only, inside level-1 group (2, 4)
    levels, passes = mips.mip_chain(eta, chi, 3, 0.01, 0.01, chi_ds_min=0.0)
    lev_b2 = mips.block_levels(passes, mips.block_empty(eta, chi, 16), 16, 2)
    assert lev_b2.shape == (2, 1, 1)
    assert lev_b2[0, 0, 0] == 0 and lev_b2[1, 0, 0] == 3
    lev_b1 = mips.block_levels(passes, mips.block_empty(eta, chi, 16), 16, 1)
    assert list(lev_b1[:, 0, 0]) == [3, 0, 3]


def test_empty_blocks_and_probe_set():
    eta = np.zeros((1, 32, 48))
    chi = np.zeros((1, 32, 48))
    chi[0, 3, 20] = 1.0
    eta[0, 30, 47] = 0.5
    empty = mips.block_empty(eta, chi, 16)
    assert empty.tolist() == [[True, False, True], [True, True, False]]
    probes = mips.probes_of_blocks(empty, 16)
    assert probes.size == 2 * 256 and probes[0] == 16 and (probes % 48 >= 16).all()


def test_generators_are_deterministic():
    a = synth.dense_exponential(32, 32)
    b = synth.dense_exponential(32, 32)
    np.testing.assert_array_equal(a["chi"], b["chi"])
    c = synth.sparse_line_atmosphere(128, 128, n_lambda=8)
    assert abs(c["empty_block_frac"] - 0.4) < 0.04
    # top 30% of the dense model is transparent and the rest is not
    assert (a["chi"][0, 32 - 9:] == 0).all() and (a["chi"][0, :32 - 9] > 0).all()


# ------------------------------------------- distance-limited MIP levels ----

def _two_block_model():
    # 32 x 16 grid: block A (x < 16) and block B (x >= 16), both selectable at level 1,
    # with a strongly varying B so that levels 0 and 1 give different intensities
    rng = np.random.default_rng(11)
    chi = rng.uniform(0.05, 0.6, (1, 16, 32))
    eta = chi * rng.uniform(0.5, 2.0, (1, 16, 32))
    levels, _ = mips.mip_chain(eta, chi, 1, 1e9, 1e9, 0.0)
    lev = np.ones((1, 1, 2), dtype=np.int32)
    return eta, chi, levels, lev


def test_banded_levels_reduce_to_plain_and_to_expanded():
    eta, chi, levels, lev = _two_block_model()
    dirs, w = synth.directions(8)
    probes = np.arange(32 * 16, dtype=np.int32)
    # no level above 0 allowed anywhere: the plain solution
    J0 = lc.formal_solve_banded(levels, lev, 16, 1, [1e9], dirs, w, probes)
    np.testing.assert_allclose(J0, lc.formal_solve(eta, chi, dirs, w, probes=probes), rtol=1e-13)
    # every level allowed from t = 0: the expanded-grid solution
    J1 = lc.formal_solve_banded(levels, lev, 16, 1, [0.0], dirs, w, probes)
    e2, c2 = mips.expand(levels, lev, 1)
    np.testing.assert_allclose(J1, lc.formal_solve(e2, c2, dirs, w, probes=probes), rtol=1e-13)
    assert np.abs(J1 - J0).max() > 1e-3  # the two limits differ for this model


def test_banded_level_switches_at_block_entry_distance():
    # A +x ray from cell (i, 3) enters block B at t = 15.5 - i.  With threshold 10,
    # probes with i <= 5 see B at level 1, probes with i >= 6 at level 0; block A
    # (entered at t = 0) is always at level 0.  Build the expected intensity by hand
    # from per-cell values of the chosen level.
    eta, chi, levels, lev = _two_block_model()
    e1 = np.repeat(np.repeat(levels[1][0][0], 2, 0), 2, 1)
    c1 = np.repeat(np.repeat(levels[1][1][0], 2, 0), 2, 1)
    for i in (2, 5, 6, 12):
        p = 3 * 32 + i
        _, I = lc.formal_solve_banded(levels, lev, 16, 1, [10.0], [[1.0, 0.0]], [1.0],
                                      np.array([p], np.int32), want_intensity=True)
        use1 = (15.5 - i) >= 10.0
        e_row = np.concatenate([eta[0, 3, :16], (e1 if use1 else eta[0])[3, 16:]])
        c_row = np.concatenate([chi[0, 3, :16], (c1 if use1 else chi[0])[3, 16:]])
        ref = 0.0
        for x in range(31, i - 1, -1):  # upwind from the boundary to the probe
            L = 0.5 if x == i else 1.0
            tau = c_row[x] * L
            ref = ref * math.exp(-tau) + e_row[x] / c_row[x] * (1 - math.exp(-tau))
        assert abs(I[0, 0, 0] - ref) < 1e-12 * ref
