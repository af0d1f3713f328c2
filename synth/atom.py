"""Seeded model atmosphere and atomic data for the statistical-equilibrium workload.

Model data only (no radiative-transfer arithmetic): a 3-level hydrogen-like
atom (levels n = 1, 2, 3; lines 1-2 and 2-3; collisional coupling between all
pairs) and a stratified temperature / electron-density atmosphere with a
transparent corona above a corrugated transition height.

The paper's 5+1-level H and Ca II/III models are not available; these values
stand in for them.  Level energies follow the Rydberg formula
E_n = 13.598 eV (1 - 1/n^2); statistical weights g_n = 2 n^2; the Einstein A
values of Lyman alpha (4.6986e8 /s) and Balmer alpha (4.4101e7 /s) are the
standard tabulated hydrogen values (NIST Atomic Spectra Database); the
effective collision strengths are round synthetic numbers.
"""

from __future__ import annotations

import numpy as np

from .atmospheres import SEED_BASE, _transition_height, lognormal_field

RYDBERG_EV = 13.598434
EV_ERG = 1.602176634e-12


def three_level_atom():
    """Atomic data as plain arrays (cgs / eV)."""
    n = np.array([1, 2, 3])
    energy_ev = RYDBERG_EV * (1.0 - 1.0 / n.astype(np.float64) ** 2)
    return {
        "energy_ev": energy_ev,                      # level energies above ground
        "g": 2.0 * n.astype(np.float64) ** 2,        # statistical weights
        # radiative lines: (lower, upper, A_ul [1/s], rest wavelength [nm])
        "lines": [(0, 1, 4.6986e8, 121.5668), (1, 2, 4.4101e7, 656.2819)],
        # effective collision strengths Upsilon_ij (i < j), all pairs
        "upsilon": {(0, 1): 0.5, (0, 2): 0.1, (1, 2): 2.0},
        "mass_amu": 1.00794,
    }


def populations_atmosphere(nx: int = 2048, nz: int = 2048, block: int = 16, empty_frac: float = 0.4,
                           seed: int = SEED_BASE + 4, t_range=(5e3, 1e5), ne_range=(1e9, 1e17),
                           sigma: float = 0.5, corr: float = 4.0, cell_cm: float = 1e6,
                           h_to_e: float = 10.0):
    """Stratified temperature and electron density below a corrugated transition.

    Below the transition height (``empty_frac`` of the blocks lie wholly above it),
    log T falls linearly with depth from ``t_range[1]`` at the transition to
    ``t_range[0]`` at the bottom, log n_e rises linearly from ``ne_range[0]`` to
    ``ne_range[1]``; both carry lognormal noise (sigma, corr).  The hydrogen
    density is ``h_to_e`` x n_e.  Above the transition every field is zero.
    Returns float32 fields ``[nz][nx]`` and the cell size in cm.
    """
    rng = np.random.default_rng(seed)
    z_tr, frac = _transition_height(nx, nz, block, empty_frac, rng)
    z = np.arange(nz, dtype=np.float64) + 0.5
    depth = z_tr[None, :] - z[:, None]
    inside = depth > 0.0
    dmax = float(np.max(z_tr))
    f = np.clip(depth / max(dmax, 1.0), 0.0, 1.0)   # 0 at the transition, 1 at the bottom
    lt = np.log(t_range[1]) + (np.log(t_range[0]) - np.log(t_range[1])) * f
    ln_e = np.log(ne_range[0]) + (np.log(ne_range[1]) - np.log(ne_range[0])) * f
    temp = np.exp(lt) * lognormal_field((nz, nx), 0.2 * sigma, corr, rng)
    temp = np.clip(temp, t_range[0], t_range[1])
    ne = np.exp(ln_e) * lognormal_field((nz, nx), sigma, corr, rng)
    temp = np.where(inside, temp, 0.0)
    ne = np.where(inside, ne, 0.0)
    return {
        "temperature": temp.astype(np.float32),
        "ne": ne.astype(np.float32),
        "nh": (h_to_e * ne).astype(np.float32),
        "cell_cm": float(cell_cm),
        "empty_block_frac": frac,
        "block": block,
    }


def line_wavelength_grid(n_per_line: int = 40, n_cont: int = 16, half_width_doppler: float = 4.0,
                         t_ref: float = 1e4):
    """Wavelength sample points (nm) and their transition tags.

    Each line gets ``n_per_line`` points uniformly over +-``half_width_doppler``
    Doppler widths at ``t_ref``; ``n_cont`` continuum points lie between the lines.
    Returns ``(lam_nm, line_index)`` with line_index = -1 for continuum points.
    """
    atom = three_level_atom()
    k_b, c, amu = 1.380649e-16, 2.99792458e10, 1.66053906660e-24
    lam, tag = [], []
    for li, (_, _, _, lam0) in enumerate(atom["lines"]):
        vth = np.sqrt(2.0 * k_b * t_ref / (atom["mass_amu"] * amu))
        dld = lam0 * vth / c
        lam.append(lam0 + half_width_doppler * dld * np.linspace(-1.0, 1.0, n_per_line))
        tag.append(np.full(n_per_line, li))
    lam.append(np.geomspace(200.0, 600.0, n_cont))
    tag.append(np.full(n_cont, -1))
    return np.concatenate(lam), np.concatenate(tag).astype(np.int32)
