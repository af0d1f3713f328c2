"""Seeded synthetic 3D inputs: a quadrature over the sphere and a sparse static
line atmosphere on a grid of 8^3 blocks.

Arrays are indexed ``[z][y][x]`` (x fastest); z is the vertical axis, x and y
horizontal.  Fields are float32, the rounding both the oracle and the CUDA path
start from.  Nothing here evaluates the radiative-transfer method.
"""

from __future__ import annotations

import numpy as np

from .atmospheres import SEED_BASE, gaussian_field, lognormal_field, smooth_uniform_field


def directions3(n_azimuth: int = 16, n_inclination: int = 4, offset: float = 0.5):
    """Product quadrature over the unit sphere.

    Azimuths phi_a = 2 pi (a + offset) / n_azimuth in the x-z plane, times
    Gauss-Legendre nodes mu_q (weights g_q, sum 2) in the direction cosine along
    y: d = (sqrt(1 - mu^2) cos phi, mu, sqrt(1 - mu^2) sin phi), w = g_q / (2 n_azimuth),
    so the weights sum to 1 (J is the angle average).  Returns float32
    ``(dirs[n][3], weights[n])``, inclination-major.
    """
    mu, g = np.polynomial.legendre.leggauss(n_inclination)
    a = np.arange(n_azimuth, dtype=np.float64)
    phi = 2.0 * np.pi * (a + offset) / n_azimuth
    s = np.sqrt(1.0 - mu * mu)
    dirs = np.stack([(s[:, None] * np.cos(phi)[None, :]).reshape(-1),
                     np.repeat(mu, n_azimuth),
                     (s[:, None] * np.sin(phi)[None, :]).reshape(-1)], axis=1)
    w = np.repeat(g / (2.0 * n_azimuth), n_azimuth)
    return dirs.astype(np.float32), w.astype(np.float32)


def _transition_height3(nx, ny, nz, block, empty_frac, rng):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    amp = nz / 256.0
    phase = rng.uniform(0.0, 2.0 * np.pi, 2)
    shape = amp * (10.0 * np.sin(2.0 * np.pi * x / 96.0 + phase[0])[None, :]
                   + 6.0 * np.sin(2.0 * np.pi * y / 53.0 + phase[1])[:, None]) \
        + 2.0 * amp * gaussian_field((ny, nx), 6.0, rng)                      # [y][x]
    nbx, nby, nbz = nx // block, ny // block, nz // block
    col_max = shape.reshape(nby, block, nbx, block).max(axis=(1, 3))           # [by][bx]
    bottoms = np.arange(nbz) * block + 0.5

    def frac(z0):
        return float((bottoms[None, None, :] >= (z0 + col_max)[:, :, None]).mean())

    lo, hi = -float(shape.max()) - 1.0, float(nz) + float(-shape.min()) + 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if frac(mid) > empty_frac:
            lo = mid
        else:
            hi = mid
    z0 = lo if abs(frac(lo) - empty_frac) <= abs(frac(hi) - empty_frac) else hi
    return z0 + shape, frac(z0)


def sparse_line_atmosphere3(nx: int = 128, ny: int = 128, nz: int = 128, block: int = 8, n_lambda: int = 16,
                            empty_frac: float = 0.4, seed: int = SEED_BASE + 30, sigma: float = 0.5,
                            corr: float = 3.0, ratio_range=(1e2, 1e5), dld_range=(1.0, 3.0)):
    """3D sparse block model with a continuum plus one line (static medium).

    The 3D counterpart of ``sparse_line_atmosphere``: below a corrugated
    transition surface ``z_tr(x, y)`` (tuned so that ``empty_frac`` of the 8^3
    blocks lie wholly above it) ``chi_c = 1e-3 exp(d / H) LN(sigma, corr)`` with
    depth d and scale height H = nz / 16 (the same optical-depth range as the 2D
    model at any height); above it every quantity is zero.  Line ratio and
    Doppler width are smooth fields; ``dlam`` is centred on the line, one grid
    unit apart.  Returns float32 fields ``[nz][ny][nx]`` plus ``dlam``.
    """
    if nx % block or ny % block or nz % block:
        raise ValueError("model extent must be a whole number of blocks")
    rng = np.random.default_rng(seed)
    z_tr, frac = _transition_height3(nx, ny, nz, block, empty_frac, rng)
    x = np.arange(nx, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    depth = z_tr[None, :, :] - z[:, None, None]
    inside = depth > 0.0
    H = nz / 16.0
    ln = lognormal_field((nz, ny, nx), sigma, corr, rng)
    chi_c = np.where(inside, 1e-3 * np.exp(np.minimum(depth, 60.0 * H) / H) * ln, 0.0)
    d_pos = np.maximum(depth, 0.0)
    s_c = np.where(inside, 1.0 + d_pos / (nz / 4.0)
                   + 0.5 * np.sin(2.0 * np.pi * x / 32.0)[None, None, :] * np.exp(-d_pos / 10.0), 0.0)
    s_l = np.where(inside, s_c * (0.3 + 0.7 * (1.0 - np.exp(-d_pos / 6.0))), 0.0)
    u1 = smooth_uniform_field((nz, ny, nx), 12.0, rng)
    u2 = smooth_uniform_field((nz, ny, nx), 12.0, rng)
    lr0, lr1 = np.log10(ratio_range[0]), np.log10(ratio_range[1])
    ratio = 10.0 ** (lr0 + (lr1 - lr0) * u1)
    dld = dld_range[0] + (dld_range[1] - dld_range[0]) * u2
    dlam = (np.arange(n_lambda, dtype=np.float64) - 0.5 * (n_lambda - 1)).astype(np.float32)
    return {"chi_c": chi_c.astype(np.float32), "s_c": s_c.astype(np.float32), "s_l": s_l.astype(np.float32),
            "ratio": ratio.astype(np.float32), "dld": dld.astype(np.float32), "dlam": dlam,
            "z_tr": z_tr.astype(np.float32), "empty_block_frac": frac, "block": block}


def random_medium3(nx: int, ny: int, nz: int, n_lambda: int, seed: int = SEED_BASE + 130,
                   log_chi_range=(-4.0, 1.5), corr: float = 2.0, zero_frac: float = 0.1,
                   emitter_frac: float = 0.02):
    """3D multi-wavelength test medium (the 3D form of ``random_medium``): per
    wavelength, log10 chi a correlated field over ``log_chi_range``, S lognormal
    around 1, a ``zero_frac`` share of empty cells and an ``emitter_frac`` share
    of transparent emitters.  Returns float32 ``eta``, ``chi`` ``[L][nz][ny][nx]``."""
    rng = np.random.default_rng(seed)
    lo, hi = log_chi_range
    shp = (nz, ny, nx)
    eta = np.empty((n_lambda,) + shp, dtype=np.float32)
    chi = np.empty((n_lambda,) + shp, dtype=np.float32)
    zero = rng.random(shp) < zero_frac
    emit = (~zero) & (rng.random(shp) < emitter_frac)
    for l in range(n_lambda):
        c = 10.0 ** (lo + (hi - lo) * smooth_uniform_field(shp, corr, rng))
        s = lognormal_field(shp, 0.5, corr, rng)
        c = np.where(zero | emit, 0.0, c).astype(np.float32)
        e = np.where(zero, 0.0, np.where(emit, 0.05 * s, c.astype(np.float64) * s))
        chi[l] = c
        eta[l] = e.astype(np.float32)
    return {"eta": eta, "chi": chi}
