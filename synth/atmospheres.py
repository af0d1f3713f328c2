"""Seeded synthetic model atmospheres (2D, x horizontal, z vertical, unit cells).

Arrays are indexed ``[z][x]`` (row ``j`` has cell-centre height ``z = j + 0.5``,
row 0 at the bottom).  Every field is returned as float32: that rounding is the
input both the oracle (which widens it to float64) and the CUDA path see.

The workloads follow the synthetic stand-ins for the paper's solar models
(the paper's KHI prominence snapshot and atomic data are not available):

* ``dense_exponential``: an exponentially stratified, lognormally perturbed
  opacity with a smooth source function and a transparent top 30% of rows,
  single wavelength.
* ``sparse_line_atmosphere``: material below a corrugated transition height,
  zero-opacity corona above it (so whole blocks are empty), a stratified
  continuum plus one line with Gaussian-shaped opacity whose strength and
  Doppler width vary smoothly over the model.

Nothing here evaluates the radiative-transfer method itself: line profiles,
emissivity/opacity sums, traversal and mipmapping live on either side.
"""

from __future__ import annotations

import numpy as np
from scipy.special import ndtr

SEED_BASE = 2511_08498


def _gaussian_filter_fft(white: np.ndarray, corr: float) -> np.ndarray:
    """Periodic Gaussian smoothing (standard deviation ``corr`` cells) of a white field."""
    freqs = [np.fft.fftfreq(n) for n in white.shape]
    k2 = np.zeros(white.shape)
    for ax, f in enumerate(freqs):
        shp = [1] * white.ndim
        shp[ax] = -1
        k2 = k2 + f.reshape(shp) ** 2
    transfer = np.exp(-2.0 * np.pi ** 2 * corr ** 2 * k2)
    g = np.fft.ifftn(np.fft.fftn(white) * transfer).real
    g = g - g.mean()
    std = g.std()
    return g / std if std > 0 else g


def gaussian_field(shape, corr: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean, unit-variance, periodic Gaussian random field with correlation length ``corr``."""
    return _gaussian_filter_fft(rng.standard_normal(shape), corr)


def lognormal_field(shape, sigma: float, corr: float, rng: np.random.Generator) -> np.ndarray:
    """exp(sigma * g) for a unit-variance correlated Gaussian field g (median 1)."""
    return np.exp(sigma * gaussian_field(shape, corr, rng))


def smooth_uniform_field(shape, corr: float, rng: np.random.Generator) -> np.ndarray:
    """Correlated field with a uniform(0, 1) marginal (normal CDF of a Gaussian field)."""
    return ndtr(gaussian_field(shape, corr, rng))


def directions(n_dir: int, offset: float = 0.5):
    """Uniform in-plane quadrature: theta_k = 2*pi*(k + offset)/n_dir, weights 1/n_dir.

    Returns ``(dirs, weights)`` with ``dirs[k] = (cos theta_k, sin theta_k)`` as float32
    (x, z components) and float32 weights.  ``offset=0`` yields axis-parallel rays.
    """
    k = np.arange(n_dir, dtype=np.float64)
    th = 2.0 * np.pi * (k + offset) / n_dir
    dirs = np.stack([np.cos(th), np.sin(th)], axis=1).astype(np.float32)
    w = np.full(n_dir, 1.0 / n_dir, dtype=np.float32)
    return dirs, w


def dense_exponential(nx: int = 128, nz: int = 128, seed: int = SEED_BASE + 1,
                      chi0: float = 1e-3, scale_height: float = 16.0,
                      sigma: float = 0.5, corr: float = 4.0, top_zero_frac: float = 0.3):
    """Dense single-wavelength model.

    chi = chi0 * exp(-z/H) * LN(sigma, corr); S = 1 + 0.5 sin(2 pi x / 64) exp(-z/40);
    eta = chi * S; the top ``floor(top_zero_frac * nz)`` rows have chi = eta = 0.
    Returns float32 ``eta``, ``chi`` of shape ``[1][nz][nx]`` (wavelength-major).
    """
    rng = np.random.default_rng(seed)
    x = np.arange(nx, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    ln = lognormal_field((nz, nx), sigma, corr, rng)
    chi = chi0 * np.exp(-z / scale_height)[:, None] * ln
    src = 1.0 + 0.5 * np.sin(2.0 * np.pi * x / 64.0)[None, :] * np.exp(-z / 40.0)[:, None]
    n_top = int(np.floor(top_zero_frac * nz))
    if n_top > 0:
        chi[nz - n_top:, :] = 0.0
    chi32 = chi.astype(np.float32)
    # eta is formed from the rounded chi so that eta == 0 exactly where chi == 0
    eta32 = (chi32.astype(np.float64) * src).astype(np.float32)
    return {"eta": eta32[None], "chi": chi32[None], "source": src.astype(np.float32)}


def _transition_height(nx: int, nz: int, block: int, empty_frac: float, rng: np.random.Generator):
    x = np.arange(nx, dtype=np.float64) + 0.5
    phase = rng.uniform(0.0, 2.0 * np.pi)
    noise = 5.0 * gaussian_field((nx,), 8.0, rng)
    amp = nz / 1024.0  # corrugation scales with the model height
    shape = amp * (40.0 * np.sin(2.0 * np.pi * x / 256.0) + 15.0 * np.sin(2.0 * np.pi * x / 61.0 + phase)) + noise
    nbx, nbz = nx // block, nz // block
    col_max = shape.reshape(nbx, block).max(axis=1)
    bottoms = np.arange(nbz) * block + 0.5  # lowest cell-centre height of each block row

    def frac(z0):
        return float((bottoms[None, :] >= (z0 + col_max)[:, None]).mean())

    lo, hi = -float(shape.max()) - 1.0, float(nz) + float(-shape.min()) + 1.0
    for _ in range(80):  # bisection: frac(z0) is non-increasing in z0
        mid = 0.5 * (lo + hi)
        if frac(mid) > empty_frac:
            lo = mid
        else:
            hi = mid
    z0 = lo if abs(frac(lo) - empty_frac) <= abs(frac(hi) - empty_frac) else hi
    return z0 + shape, frac(z0)


def sparse_line_atmosphere(nx: int = 1024, nz: int = 1024, block: int = 16, n_lambda: int = 32,
                           empty_frac: float = 0.4, seed: int = SEED_BASE + 2,
                           sigma: float = 0.5, corr: float = 4.0, scale_height: float = 64.0,
                           ratio_range=(1e2, 1e5), dld_range=(1.0, 3.0)):
    """Sparse block model with a continuum plus one line (static medium).

    Below the corrugated transition height ``z_tr(x)`` (tuned so that ``empty_frac`` of
    the ``block``-sized blocks lie wholly above it) the continuum opacity grows downward,
    ``chi_c = 1e-3 exp(d / H) LN(sigma, corr)`` with depth ``d = z_tr - z``; above it every
    quantity is zero.  Line parameters per cell: peak line-to-continuum opacity ratio
    ``ratio`` (log-uniform over ``ratio_range`` as a smooth field) and Doppler width
    ``dld`` in wavelength-grid units.  ``dlam`` holds the ``n_lambda`` wavelength offsets
    from line centre, spaced one grid unit apart and centred on the line.
    Returns float32 fields ``[nz][nx]`` plus ``dlam`` and bookkeeping.
    """
    if nx % block or nz % block:
        raise ValueError("model extent must be a whole number of blocks")
    rng = np.random.default_rng(seed)
    z_tr, frac = _transition_height(nx, nz, block, empty_frac, rng)
    x = np.arange(nx, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    depth = z_tr[None, :] - z[:, None]
    inside = depth > 0.0
    ln = lognormal_field((nz, nx), sigma, corr, rng)
    chi_c = np.where(inside, 1e-3 * np.exp(np.minimum(depth, 60.0 * scale_height) / scale_height) * ln, 0.0)
    d_pos = np.maximum(depth, 0.0)
    s_c = np.where(inside, 1.0 + d_pos / 256.0
                   + 0.5 * np.sin(2.0 * np.pi * x / 64.0)[None, :] * np.exp(-d_pos / 40.0), 0.0)
    s_l = np.where(inside, s_c * (0.3 + 0.7 * (1.0 - np.exp(-d_pos / 24.0))), 0.0)
    u1 = smooth_uniform_field((nz, nx), 32.0, rng)
    u2 = smooth_uniform_field((nz, nx), 32.0, rng)
    lr0, lr1 = np.log10(ratio_range[0]), np.log10(ratio_range[1])
    ratio = 10.0 ** (lr0 + (lr1 - lr0) * u1)
    dld = dld_range[0] + (dld_range[1] - dld_range[0]) * u2
    dlam = (np.arange(n_lambda, dtype=np.float64) - 0.5 * (n_lambda - 1)).astype(np.float32)
    return {
        "chi_c": chi_c.astype(np.float32),
        "s_c": s_c.astype(np.float32),
        "s_l": s_l.astype(np.float32),
        "ratio": ratio.astype(np.float32),
        "dld": dld.astype(np.float32),
        "dlam": dlam,
        "z_tr": z_tr.astype(np.float32),
        "empty_block_frac": frac,
        "block": block,
    }


def random_medium(nx: int, nz: int, n_lambda: int, seed: int = SEED_BASE + 100,
                  log_chi_range=(-4.0, 1.5), corr: float = 3.0,
                  zero_frac: float = 0.1, emitter_frac: float = 0.02):
    """Multi-wavelength test medium with structure at every scale the solvers meet.

    Per wavelength, log10 chi is a correlated field spread over ``log_chi_range``
    (optical depths per cell from ~1e-4 to ~30); S is lognormal around 1.  A
    ``zero_frac`` share of cells is empty (eta = chi = 0) and an ``emitter_frac``
    share is a transparent emitter (chi = 0, eta > 0).  Returns float32
    ``eta``, ``chi`` of shape ``[n_lambda][nz][nx]``.
    """
    rng = np.random.default_rng(seed)
    lo, hi = log_chi_range
    eta = np.empty((n_lambda, nz, nx), dtype=np.float32)
    chi = np.empty((n_lambda, nz, nx), dtype=np.float32)
    zero = rng.random((nz, nx)) < zero_frac
    emit = (~zero) & (rng.random((nz, nx)) < emitter_frac)
    for l in range(n_lambda):
        u = smooth_uniform_field((nz, nx), corr, rng)
        c = 10.0 ** (lo + (hi - lo) * u)
        s = lognormal_field((nz, nx), 0.5, corr, rng)
        c = np.where(zero | emit, 0.0, c).astype(np.float32)
        e = (c.astype(np.float64) * s)
        e = np.where(emit, 0.05 * s, e)
        e = np.where(zero, 0.0, e)
        chi[l] = c
        eta[l] = e.astype(np.float32)
    return {"eta": eta, "chi": chi}


C_KMS = 299792.458


def dynamic_line_atmosphere(nx: int = 2048, nz: int = 1024, block: int = 16, n_lambda: int = 64,
                            empty_frac: float = 0.4, seed: int = SEED_BASE + 3, sigma: float = 0.5,
                            corr: float = 4.0, scale_height: float = 64.0, ratio_range=(1e2, 1e5),
                            vmax: float = 50.0, vth_range=(5.0, 10.0), damping_range=(1e-3, 1e-1),
                            lambda0_nm: float = 656.28):
    """Moving-medium model: continuum + one Voigt line with a line-of-sight velocity field.

    Same transition/continuum construction as ``sparse_line_atmosphere``.  Per cell:
    velocity (vx, vz) in km/s = three seeded smooth Fourier modes plus two tanh shear
    layers, rescaled so |v| <= ``vmax``; thermal (Doppler) width v_th in km/s, smooth
    uniform over ``vth_range``; damping a, log-uniform over ``damping_range`` as a smooth
    field; line strength ``chi_star`` (per cell, per km/s) = r chi_c sqrt(pi) v_th, so that
    the undamped line-centre opacity is r chi_c with r log-uniform over ``ratio_range``;
    ``eta_star`` = chi_star S_l.  Wavelengths are velocity offsets ``dv`` (km/s) from the
    rest wavelength ``lambda0_nm``, uniform over +-(vmax + 3 max v_th).
    """
    if nx % block or nz % block:
        raise ValueError("model extent must be a whole number of blocks")
    rng = np.random.default_rng(seed)
    z_tr, frac = _transition_height(nx, nz, block, empty_frac, rng)
    x = np.arange(nx, dtype=np.float64) + 0.5
    z = np.arange(nz, dtype=np.float64) + 0.5
    X, Z = np.meshgrid(x, z)
    depth = z_tr[None, :] - z[:, None]
    inside = depth > 0.0
    ln = lognormal_field((nz, nx), sigma, corr, rng)
    chi_c = np.where(inside, 1e-3 * np.exp(np.minimum(depth, 60.0 * scale_height) / scale_height) * ln, 0.0)
    d_pos = np.maximum(depth, 0.0)
    s_c = np.where(inside, 1.0 + d_pos / 256.0 + 0.5 * np.sin(2.0 * np.pi * X / 64.0) * np.exp(-d_pos / 40.0), 0.0)
    s_l = np.where(inside, s_c * (0.3 + 0.7 * (1.0 - np.exp(-d_pos / 24.0))), 0.0)
    vel = []
    for _ in range(2):
        f = np.zeros((nz, nx))
        for _m in range(3):
            kx, kz = rng.uniform(-4, 4, 2) * 2 * np.pi / np.array([nx, nz])
            f += rng.uniform(0.3, 1.0) * np.sin(kx * X + kz * Z + rng.uniform(0, 2 * np.pi))
        vel.append(f)
    z1, z2 = rng.uniform(0.2, 0.8, 2) * nz
    vel[0] = vel[0] + 1.5 * np.tanh((Z - z1) / 6.0) - 1.5 * np.tanh((Z - z2) / 6.0)
    vx, vz = vel
    mag = np.sqrt(vx * vx + vz * vz)
    scale = vmax / max(float(mag.max()), 1e-30)
    vx, vz = vx * scale, vz * scale
    vth = vth_range[0] + (vth_range[1] - vth_range[0]) * smooth_uniform_field((nz, nx), 32.0, rng)
    la0, la1 = np.log10(damping_range[0]), np.log10(damping_range[1])
    damping = 10.0 ** (la0 + (la1 - la0) * smooth_uniform_field((nz, nx), 32.0, rng))
    lr0, lr1 = np.log10(ratio_range[0]), np.log10(ratio_range[1])
    ratio = 10.0 ** (lr0 + (lr1 - lr0) * smooth_uniform_field((nz, nx), 32.0, rng))
    chi_star = ratio * chi_c * np.sqrt(np.pi) * vth
    half = vmax + 3.0 * vth_range[1]
    dv = np.linspace(-half, half, n_lambda)
    f32 = lambda a: np.where(inside, a, 0.0).astype(np.float32)
    return {
        "chi_star": f32(chi_star), "eta_star": f32(chi_star * s_l), "damping": f32(damping),
        "vth": f32(vth), "vx": f32(vx), "vz": f32(vz), "chi_c": f32(chi_c), "eta_c": f32(chi_c * s_c),
        "dv": dv.astype(np.float32), "lambda0_nm": float(lambda0_nm), "c_kms": C_KMS,
        "empty_block_frac": frac, "block": block,
    }


def batch_specs(n_atm: int = 24, seed: int = SEED_BASE + 5, sizes=((256, 256), (2048, 1024)),
                n_lambda=(16, 96), n_dir=(32, 128), empty=(0.1, 0.7), scale: float = 1.0):
    """Seeded list of independent atmosphere specs for the batched workload.

    Side lengths are drawn log-uniformly between the two corner sizes (multiples of
    64, times ``scale``), wavelength counts and direction counts uniformly in
    multiples of 8, empty-block fractions uniformly.  Each spec carries its own seed
    for ``sparse_line_atmosphere``.
    """
    rng = np.random.default_rng(seed)
    (x0, z0), (x1, z1) = sizes
    out = []
    for a in range(n_atm):
        nx = int(round(np.exp(rng.uniform(np.log(x0), np.log(x1))) * scale / 64)) * 64
        nz = int(round(np.exp(rng.uniform(np.log(z0), np.log(z1))) * scale / 64)) * 64
        out.append({"nx": max(nx, 64), "nz": max(nz, 64),
                    "n_lambda": int(rng.integers(n_lambda[0] // 8, n_lambda[1] // 8 + 1)) * 8,
                    "n_dir": int(rng.integers(n_dir[0] // 8, n_dir[1] // 8 + 1)) * 8,
                    "empty_frac": float(rng.uniform(*empty)), "seed": int(seed * 100 + a)})
    return out


def rc_directions(n0: int = 4, n_cascades: int = 6):
    """Direction sets of radiance cascades with branching factor 2: cascade i has
    n0 * 4^i in-plane directions theta_k = 2*pi*(k + 1/2) / (n0 * 4^i), so that
    directions 4k .. 4k+3 of cascade i + 1 split direction k of cascade i.
    Returns a list of float32 ``[n_i][2]`` arrays (x, z components); cascade 0
    equals ``directions(n0)``."""
    return [directions(n0 * 4 ** i)[0] for i in range(n_cascades)]
