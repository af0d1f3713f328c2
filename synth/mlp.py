"""Seeded inputs of the learned profile surrogate: sample points and initial weights.

Random draws only (no profile evaluation, no network arithmetic).  Sample
ranges follow the dynamic-line workload: wavelength offsets within +-16 Doppler
widths (+-80 km/s at a 5 km/s thermal width), projected velocities within +-10
Doppler widths (+-50 km/s), damping log-uniform in [1e-3, 1e-1].
"""

from __future__ import annotations

import numpy as np

from .atmospheres import SEED_BASE

X_MAX = 16.0
U_MAX = 10.0
LOG10_A = (-3.0, -1.0)
HIDDEN = 64
N_PARAMS = HIDDEN * 3 + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def voigt_samples(n: int, seed: int = SEED_BASE + 900, core_fraction: float = 0.0, core_width: float = 2.5):
    """[n][3] float32 (x, a, u): x, u uniform, log10 a uniform.  A fraction
    ``core_fraction`` of the samples instead draws x - u from a normal of width
    ``core_width`` Doppler widths (clipped to the x range), over-sampling the line
    core where the profile changes fastest."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-X_MAX, X_MAX, n)
    a = 10.0 ** rng.uniform(LOG10_A[0], LOG10_A[1], n)
    u = rng.uniform(-U_MAX, U_MAX, n)
    core = rng.uniform(0.0, 1.0, n) < core_fraction
    d = rng.normal(0.0, core_width, n)
    x = np.where(core, np.clip(u + d, -X_MAX, X_MAX), x)
    return np.ascontiguousarray(np.stack([x, a, u], axis=1).astype(np.float32))


def initial_params(seed: int = SEED_BASE + 901, scale: float = 1.0):
    """Float32 parameter vector in the library's layout (W1, b1, W2, b2, w3, b3):
    weights normal with variance 2 / fan_in (He initialisation) times ``scale``,
    biases zero except the output bias, set to -4 (about the mean ln H of the
    sample ranges)."""
    rng = np.random.default_rng(seed)
    H = HIDDEN
    W1 = rng.normal(0.0, np.sqrt(2.0 / 3.0), (H, 3)) * scale
    W2 = rng.normal(0.0, np.sqrt(2.0 / H), (H, H)) * scale
    w3 = rng.normal(0.0, np.sqrt(2.0 / H), H) * scale
    p = np.concatenate([W1.reshape(-1), np.zeros(H), W2.reshape(-1), np.zeros(H), w3, [-4.0]])
    assert p.size == N_PARAMS
    return p.astype(np.float32)


def random_params(seed: int, scale: float = 0.5):
    """Parameters with random biases as well (for parity tests)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(0.0, scale, N_PARAMS)).astype(np.float32)
