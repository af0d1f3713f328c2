"""Pins of the 3D float64 oracle against facts that do not come from it: an exact
rational cell walk (a different algorithm from the oracle's sorted plane
crossings), closed forms of the segment count and of the uniform medium,
brute-force sub-stepping, the reduction to the (separately pinned) 2D oracle,
invariance under a relabelling of the axes, hand-computed Morton codes and
IoD values, and the 3D MIP storage factor the paper prints (Section 2.1).
"""

import math
from fractions import Fraction as F

import numpy as np
import pytest

import synth
from oracle import lc, lc3, mips, mips3


# ---------------------------------------------------------------- geometry ----

def exact_cells3(shape, o, d):
    """Cell-by-cell walk in exact rational arithmetic: [(cell, length_in_t)], t_exit."""
    n = shape
    o = [F(v) for v in o]
    d = [F(v) for v in d]

    def exit_t(a):
        if d[a] > 0:
            return (n[a] - o[a]) / d[a]
        if d[a] < 0:
            return (0 - o[a]) / d[a]
        return None

    tex = min(t for t in (exit_t(a) for a in range(3)) if t is not None)
    c = [math.floor(v) for v in o]
    t = F(0)
    out = []
    while t < tex:
        nxt_ax = []
        for a in range(3):
            if d[a] > 0:
                nxt_ax.append((c[a] + 1 - o[a]) / d[a])
            elif d[a] < 0:
                nxt_ax.append((c[a] - o[a]) / d[a])
            else:
                nxt_ax.append(None)
        nxt = min(v for v in nxt_ax + [tex] if v is not None)
        if nxt > t:
            out.append(((c[2] * n[1] + c[1]) * n[0] + c[0], nxt - t))
        if nxt == tex:
            break
        for a in range(3):
            if nxt_ax[a] is not None and nxt_ax[a] == nxt:
                c[a] += 1 if d[a] > 0 else -1
        t = nxt
    return out, tex


GEOM3 = [
    ((5, 4, 3), (F(1, 2), F(1, 2), F(1, 2)), (1, 1, 1)),            # through cube corners
    ((6, 5, 7), (F(11, 2), F(1, 2), F(13, 2)), (-1, 1, -1)),
    ((6, 6, 6), (F(5, 2), F(3, 2), F(1, 2)), (F(2, 3), F(1, 3), F(2, 3))),
    ((7, 4, 5), (F(3, 2), F(5, 2), F(7, 2)), (F(-6, 7), F(2, 7), F(-3, 7))),
    ((9, 3, 4), (F(3, 2), F(1, 2), F(5, 2)), (1, 0, 0)),            # axis parallel
    ((3, 9, 4), (F(1, 2), F(15, 2), F(3, 2)), (0, -1, 0)),
    ((4, 4, 9), (F(1, 2), F(5, 2), F(1, 2)), (0, 0, 1)),
    ((8, 8, 8), (F(1, 2), F(13, 2), F(7, 2)), (F(8, 17), F(-15, 17), 0)),  # in a y-x plane
    ((5, 9, 6), (F(9, 2), F(1, 2), F(3, 2)), (-2, 3, 1)),           # non-unit direction
]


@pytest.mark.parametrize("shape,o,d", GEOM3)
def test_segments_match_exact_rational_walk(shape, o, d):
    exact, tex = exact_cells3(shape, o, d)
    cells, lens = lc3.ray_segments(shape, [float(v) for v in o], [float(v) for v in d])
    assert [c for c, _ in exact] == list(cells)
    np.testing.assert_allclose(lens, [float(L) for _, L in exact], rtol=0, atol=1e-12)
    assert abs(lens.sum() - float(tex)) < 1e-12


def test_segment_lengths_sum_to_exit_distance():
    dirs, _ = synth.directions3(8, 4)
    shape = (7, 6, 5)
    for c in [(0, 0, 0), (3, 2, 4), (6, 5, 4), (1, 4, 2)]:
        o = [v + 0.5 for v in c]
        for d in dirs.astype(np.float64):
            _, lens = lc3.ray_segments(shape, o, d)
            tex = min((shape[a] - o[a]) / d[a] if d[a] > 0 else (-o[a] / d[a] if d[a] < 0 else np.inf)
                      for a in range(3))
            assert abs(lens.sum() - tex) < 1e-10


def test_axis_parallel_segment_count_closed_form():
    # Six axis-parallel rays from every cell centre: toward +x from column i the
    # ray crosses nx - i cells and toward -x i + 1, so the pair adds nx + 1 per
    # cell; over all cells the total is N (nx + ny + nz + 3), N = nx ny nz.
    nx, ny, nz = 5, 4, 6
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    probes = np.arange(nx * ny * nz, dtype=np.int32)
    assert lc3.count_segments((nx, ny, nz), dirs, probes) == nx * ny * nz * (nx + ny + nz + 3)


# ------------------------------------------------------- closed-form RTE ----

def _texit3(shape, o, d):
    return min((shape[a] - o[a]) / d[a] if d[a] > 0 else (-o[a] / d[a] if d[a] < 0 else np.inf)
               for a in range(3))


def _origin(p, shape):
    nx, ny, _ = shape
    return (p % nx + 0.5, (p // nx) % ny + 0.5, p // (nx * ny) + 0.5)


def test_uniform_medium_closed_form():
    shape = (9, 7, 8)
    chi0, S = 0.29, 1.75
    eta = np.full((1, 8, 7, 9), chi0 * S)
    chi = np.full((1, 8, 7, 9), chi0)
    dirs, w = synth.directions3(8, 4)
    d64 = dirs.astype(np.float64)
    for ibc in (0.0, 2.2):
        J, I = lc3.formal_solve(eta, chi, d64, w, i_bc=ibc, want_intensity=True)
        for p in [0, 40, 9 * 7 * 8 - 1, 211]:
            o = _origin(p, shape)
            for k in range(d64.shape[0]):
                tau = chi0 * _texit3(shape, o, d64[k])
                ref = S * (1 - math.exp(-tau)) + ibc * math.exp(-tau)
                assert abs(I[0, k, p] - ref) <= 1e-13 * max(1.0, abs(ref))
            assert abs(J[0, p] - np.dot(np.asarray(w, np.float64), I[0, :, p])) < 1e-13


def test_transparent_medium_and_weights():
    shape = (6, 5, 4)
    dirs, w = synth.directions3(6, 2)
    zero = np.zeros((1, 4, 5, 6))
    J = lc3.formal_solve(zero, zero, dirs, w, i_bc=3.25)
    np.testing.assert_allclose(J, 3.25 * np.asarray(w, np.float64).sum(), rtol=1e-15)
    eta = np.full((1, 4, 5, 6), 0.6)
    _, I = lc3.formal_solve(eta, zero, dirs, w, i_bc=1.0, want_intensity=True)
    d64 = dirs.astype(np.float64)
    for p in [0, 37, 119]:
        o = _origin(p, shape)
        for k in range(d64.shape[0]):
            assert abs(I[0, k, p] - (1.0 + 0.6 * _texit3(shape, o, d64[k]))) < 1e-12


def _substep3(eta, chi, o, d, ibc, h):
    nz, ny, nx = eta.shape
    tex = _texit3((nx, ny, nz), o, d)
    n = int(math.ceil(tex / h))
    I = ibc
    for s in range(n - 1, -1, -1):
        t0, t1 = s * h, min((s + 1) * h, tex)
        tm = 0.5 * (t0 + t1)
        i = min(max(int(math.floor(o[0] + tm * d[0])), 0), nx - 1)
        j = min(max(int(math.floor(o[1] + tm * d[1])), 0), ny - 1)
        k = min(max(int(math.floor(o[2] + tm * d[2])), 0), nz - 1)
        x, e, L = chi[k, j, i], eta[k, j, i], t1 - t0
        I = I * math.exp(-x * L) + e / x * (1 - math.exp(-x * L)) if x > 0 else I + e * L
    return I


def test_brute_force_substepping():
    rng = np.random.default_rng(11)
    nx, ny, nz = 5, 4, 4
    chi = rng.uniform(0.0, 2.0, (nz, ny, nx))
    chi[1, 2, 3] = 0.0
    S = rng.uniform(0.5, 3.0, (nz, ny, nx))
    eta = chi * S
    eta[1, 2, 3] = 0.4
    dirs = rng.normal(size=(5, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    _, I = lc3.formal_solve(eta[None], chi[None], dirs, np.ones(5), i_bc=0.25, want_intensity=True)
    for p in [0, 27, 79]:
        o = _origin(p, (nx, ny, nz))
        for k in range(5):
            ref = _substep3(eta, chi, o, dirs[k], 0.25, 2e-4)
            assert abs(I[0, k, p] - ref) < 3e-3 * max(ref, 1e-3)


def test_reduces_to_the_2d_oracle_on_a_one_cell_thick_grid():
    # ny = 1 and d_y = 0: every ray stays in the x-z plane, so the 3D solve is the
    # (separately pinned) 2D solve with cell j * nx + i.
    m = synth.random_medium(12, 10, 3, seed=synth.SEED_BASE + 131)
    eta2, chi2 = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    d2, w = synth.directions(16)
    d3 = np.stack([d2[:, 0], np.zeros(16, np.float32), d2[:, 1]], 1)
    J2 = lc.formal_solve(eta2, chi2, d2, w, i_bc=0.3)
    J3 = lc3.formal_solve(eta2[:, :, None, :], chi2[:, :, None, :], d3, w, i_bc=0.3)
    np.testing.assert_allclose(J3, J2, rtol=1e-13, atol=0)
    # the same plane as a y-z slab (nx = 1, rays in y-z): relabel x -> y
    d3b = np.stack([np.zeros(16, np.float32), d2[:, 0], d2[:, 1]], 1)
    J3b = lc3.formal_solve(eta2[:, :, :, None], chi2[:, :, :, None], d3b, w, i_bc=0.3)
    np.testing.assert_allclose(J3b, J2, rtol=1e-13, atol=0)


def test_axis_relabelling_invariance():
    m = synth.random_medium3(6, 5, 4, 2, seed=synth.SEED_BASE + 132)
    eta, chi = m["eta"].astype(np.float64), m["chi"].astype(np.float64)
    dirs, w = synth.directions3(6, 4)
    J = lc3.formal_solve(eta, chi, dirs, w, i_bc=0.1).reshape(2, 4, 5, 6)
    # swap the x and z axes of the grid and of every direction
    et, ct = eta.transpose(0, 3, 2, 1), chi.transpose(0, 3, 2, 1)
    Jt = lc3.formal_solve(np.ascontiguousarray(et), np.ascontiguousarray(ct), dirs[:, ::-1].copy(), w,
                          i_bc=0.1).reshape(2, 6, 5, 4)
    np.testing.assert_allclose(Jt.transpose(0, 3, 2, 1), J, rtol=1e-12, atol=0)


# ----------------------------------------------- MIP chain and block map ----

def test_3d_mip_storage_factor_printed_in_paper():
    # Section 2.1: the 3D MIP chain costs 1.14x MIP 0.  An 8^3 block with levels
    # 0..3 holds 512 + 64 + 8 + 1 = 585 voxels.
    assert round(585 / 512, 2) == 1.14
    rng = np.random.default_rng(1)
    e = rng.uniform(0.1, 1.0, (1, 8, 8, 8))
    levels, passes = mips3.mip_chain(e, e, 3, 1.0, 1.0)
    assert [lv[0].size for lv in levels] == [512, 64, 8, 1]
    assert len(passes) == 3


def test_morton3_by_hand():
    assert [mips3.morton3(*c) for c in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (2, 0, 0)]] == [1, 2, 4, 7, 8]
    # (3, 5, 6): bit triples (z y x) = 011, 101, 110 from bit 0 up: 3 + 5*8 + 6*64
    assert mips3.morton3(3, 5, 6) == 427
    empty = np.zeros((2, 2, 4), bool)          # nbz = 2, nby = 2, nbx = 4
    empty[0, 1, 1] = True
    active, offset = mips3.block_layout(empty)
    # Z-order over (bx, by, bz): codes of the active blocks sorted; hand-listed
    # first blocks: (0,0,0)=0, (1,0,0)=1, (0,1,0)=2, [(1,1,0) empty], (0,0,1)=4, (1,0,1)=5
    assert list(active[:5]) == [0, 1, 4, 8, 9]
    assert offset[0, 1, 1] == -1 and offset.max() == 14


def test_iod_of_a_two_valued_group_by_hand():
    # Children a (4 of them) and b (4): X = ln(g Ds); mean ln(Ds) + (ln a + ln b)/2,
    # population variance ((ln a - ln b)/2)^2.
    a, b, ds = 2.0, 0.5, 2.0
    g = np.array([a, b, a, b, b, a, a, b]).reshape(1, 2, 2, 2)
    levels, _, st = mips3.mip_chain(g, g, 1, 1.0, 1.0, stats=True)
    mu = math.log(ds) + 0.5 * (math.log(a) + math.log(b))
    var = (0.5 * (math.log(a) - math.log(b))) ** 2
    assert abs(st[0]["iod_eta"][0, 0, 0, 0] - abs(var / mu)) < 1e-14
    assert abs(levels[1][0][0, 0, 0, 0] - math.sqrt(a * b)) < 1e-15      # log mean
    lin, _ = mips3.mip_chain(g, g, 1, 1.0, 1.0, mean="linear")
    assert abs(lin[1][0][0, 0, 0, 0] - 0.5 * (a + b)) < 1e-15


def test_homogeneous_blocks_reach_level_3_and_the_levels_change_nothing():
    eta = np.full((2, 16, 8, 16), 0.7)
    chi = np.full((2, 16, 8, 16), 0.35)
    eta[:, :8, :, 8:] = 0.0                      # one empty block column
    chi[:, :8, :, 8:] = 0.0
    empty = mips3.block_empty(eta, chi, 8)
    assert empty.sum() == 1
    levels, passes = mips3.mip_chain(eta, chi, 3, 1e-3, 1e-3, mean="log")
    lev = mips3.block_levels(passes, empty, 8, 2)
    assert (lev[0][~empty] == 3).all() and (lev[0][empty] == -1).all()
    ee, ce = mips3.expand(levels, lev, 2)
    np.testing.assert_allclose(ee, eta, rtol=1e-15)
    dirs, w = synth.directions3(4, 2)
    probes = mips3.probes_of_blocks(empty, 8)
    J0 = lc3.formal_solve(eta, chi, dirs, w, probes=probes)
    Jb = lc3.formal_solve_banded(levels, lev, 8, 2, [0.0, 0.0, 0.0], dirs, w, probes)
    np.testing.assert_allclose(Jb, J0, rtol=1e-12)


def test_block_level_is_minimum_over_wavelength_batch():
    rng = np.random.default_rng(3)
    eta = np.full((3, 8, 8, 8), 1.0)
    chi = np.full((3, 8, 8, 8), 1.0)
    eta[1] = rng.uniform(0.01, 100.0, (8, 8, 8))  # wavelength 1 is very rough
    empty = mips3.block_empty(eta, chi, 8)
    _, passes = mips3.mip_chain(eta, chi, 3, 0.1, 0.1)
    assert mips3.block_levels(passes, empty, 8, 1)[:, 0, 0, 0].tolist() == [3, 0, 3]
    assert mips3.block_levels(passes, empty, 8, 2)[:, 0, 0, 0].tolist() == [0, 3]
    assert mips3.block_levels(passes, empty, 8, 4)[:, 0, 0, 0].tolist() == [0]


def test_groups_are_the_2x2x2_children():
    # Level-1 voxel (0,0,1) of an [z][y][x] = [2][2][4] grid averages cells x in {2,3}.
    a = np.arange(16, dtype=np.float64).reshape(1, 2, 2, 4) + 1.0
    lv, _ = mips3.mip_chain(a, a, 1, 1.0, 1.0, mean="linear")
    kids = a[0, 0:2, 0:2, 2:4]
    assert lv[1][0][0, 0, 0, 1] == kids.mean()
    # and the 2D oracle's reduction gives the same value on the same 8 numbers
    v, _ = mips._reduce(kids.reshape(1, 8), 2.0, "linear")
    assert v[0] == kids.mean()


def test_banded_levels_switch_at_block_entry_distance():
    # Two homogeneous blocks along x at very different values; the far block
    # is at level 3.  With band [0.5, 100, 100] a +x ray enters the far block at
    # t = 7.5 >= 0.5: level min(3, 1) = 1, which equals MIP 0 for a homogeneous
    # block; with band [100, ...] it is level 0.  Both equal the plain solve.
    eta = np.zeros((1, 8, 8, 16))
    chi = np.zeros((1, 8, 8, 16))
    chi[..., :8], eta[..., :8] = 0.2, 0.2 * 1.5
    chi[..., 8:], eta[..., 8:] = 0.9, 0.9 * 0.4
    empty = mips3.block_empty(eta, chi, 8)
    levels, passes = mips3.mip_chain(eta, chi, 3, 1e-3, 1e-3)
    lev = mips3.block_levels(passes, empty, 8, 1)
    dirs = np.array([[1.0, 0.0, 0.0]])
    probes = np.array([0], np.int32)
    ref = lc3.formal_solve(eta, chi, dirs, [1.0], probes=probes)
    for band in ([0.5, 100.0, 100.0], [100.0, 100.0, 100.0], []):
        J = lc3.formal_solve_banded(levels, lev, 8, 1, band, dirs, [1.0], probes)
        np.testing.assert_allclose(J, ref, rtol=1e-13)
    # a rough far block: the level used there changes J exactly as the band says
    rng = np.random.default_rng(9)
    chi[..., 8:] = rng.uniform(0.1, 2.0, (1, 8, 8, 8))
    eta[..., 8:] = chi[..., 8:] * 0.4
    levels, passes = mips3.mip_chain(eta, chi, 3, 1e30, 1e30)
    lev = mips3.block_levels(passes, mips3.block_empty(eta, chi, 8), 8, 1)
    assert lev[0, 0, 0, 1] == 3
    J_far0 = lc3.formal_solve_banded(levels, lev, 8, 1, [100.0], dirs, [1.0], probes)
    J_far1 = lc3.formal_solve_banded(levels, lev, 8, 1, [7.5, 100.0], dirs, [1.0], probes)
    np.testing.assert_allclose(J_far0, lc3.formal_solve(eta, chi, dirs, [1.0], probes=probes), rtol=1e-13)
    e1 = lc3.upsample(levels[1][0], 2)
    c1 = lc3.upsample(levels[1][1], 2)
    mixed_e, mixed_c = eta.copy(), chi.copy()
    mixed_e[..., 8:], mixed_c[..., 8:] = e1[..., 8:], c1[..., 8:]
    np.testing.assert_allclose(J_far1, lc3.formal_solve(mixed_e, mixed_c, dirs, [1.0], probes=probes), rtol=1e-13)
    assert abs(J_far1[0, 0] - J_far0[0, 0]) > 1e-6
