"""Pins of the float64 surrogate-network reference (oracle/mlp.py) to facts that do
not come from its own formulas: central finite differences of the loss, the
closed forms of GELU and of a network with zero weights, the bfloat16 rounding
rule on hand-chosen values, and a hand-computed one-sample network.
"""

import numpy as np
import pytest

import synth
from oracle import mlp

GROUPS = {"W1": (0, 192), "b1": (192, 256), "W2": (256, 4352), "b2": (4352, 4416), "w3": (4416, 4480),
          "b3": (4480, 4481)}


def _problem(n=48, seed=5):
    p = synth.mlp.random_params(synth.SEED_BASE + seed, scale=0.4).astype(np.float64)
    xau = synth.mlp.voigt_samples(n, seed=synth.SEED_BASE + seed + 1).astype(np.float64)
    t = np.random.default_rng(seed).normal(-4.0, 2.0, n)
    return p, xau, t


def test_gradient_matches_central_differences():
    p, xau, t = _problem()
    _, g = mlp.loss_and_grad(p, xau, t, emulate=False)
    rng = np.random.default_rng(0)
    h = 1e-6
    for name, (a, b) in GROUPS.items():
        idx = rng.choice(np.arange(a, b), size=min(12, b - a), replace=False)
        for q in idx:
            pp, pm = p.copy(), p.copy()
            pp[q] += h
            pm[q] -= h
            fd = (mlp.loss_and_grad(pp, xau, t, emulate=False)[0] - mlp.loss_and_grad(pm, xau, t, emulate=False)[0]) / (2 * h)
            assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)), (name, q, fd, g[q])


def test_gelu_closed_forms():
    assert mlp.gelu(np.float64(0.0)) == 0.0
    assert mlp.gelu_prime(np.float64(0.0)) == 0.5
    # tanh saturates: GELU(z) -> z for large z, -> 0 for large -z
    assert abs(mlp.gelu(12.0) - 12.0) < 1e-12
    assert abs(mlp.gelu(-12.0)) < 1e-12
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(fd, mlp.gelu_prime(z), atol=1e-8)
    # the tanh form at z = 1: 0.5 (1 + tanh(sqrt(2/pi) 1.044715))
    assert abs(mlp.gelu(1.0) - 0.5 * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * 1.044715))) < 1e-15


def test_zero_weight_network():
    p, xau, t = _problem(n=16)
    d = mlp.unpack(p)
    d["W1"][:] = 0.0
    d["W2"][:] = 0.0
    d["w3"][:] = 0.0
    d["b2"][:] = 0.0
    d["b3"] = 1.25
    q = mlp.pack(d)
    for emulate in (False, True):
        y = mlp.forward(q, xau, emulate=emulate)
        assert np.all(y == 1.25)
        loss, g = mlp.loss_and_grad(q, xau, t, emulate=emulate)
        assert abs(loss - np.mean((1.25 - t) ** 2)) < 1e-12
        assert abs(g[4480] - 2.0 * np.mean(1.25 - t)) < 1e-12
        # h2 = GELU(0) = 0 and w3 = 0: no gradient reaches W2, b2, w3, W1, b1
        assert not np.any(g[:4480])


def test_features_and_one_sample_by_hand():
    f = mlp.features(np.array([[16.0, 0.01, -16.0]]))
    assert np.array_equal(f, [[1.0, 0.0, -1.0]])
    # one sample, one active path: W1[0] = (1, 0, 0), W2[0][0] = 1, w3[0] = 1
    p = np.zeros(mlp.N_PARAMS)
    d = mlp.unpack(p)
    d["W1"][0, 0] = 1.0
    d["W2"][0, 0] = 1.0
    d["w3"][0] = 1.0
    q = mlp.pack(d)
    y = mlp.forward(q, np.array([[8.0, 0.01, 0.0]]), emulate=False)[0]
    z1 = 0.5
    g1 = 0.5 * z1 * (1 + np.tanh(np.sqrt(2 / np.pi) * (z1 + 0.044715 * z1 ** 3)))
    g2 = 0.5 * g1 * (1 + np.tanh(np.sqrt(2 / np.pi) * (g1 + 0.044715 * g1 ** 3)))
    assert abs(y - g2) < 1e-15


def test_bf16_rounding_rule():
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3.0 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (1 + 2^-6)
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-3.0) == -3.0
    assert mlp.bf16(0.0) == 0.0


def test_emulated_gradient_close_to_exact():
    p, xau, t = _problem(n=256, seed=9)
    _, ge = mlp.loss_and_grad(p, xau, t, emulate=True)
    _, gx = mlp.loss_and_grad(p, xau, t, emulate=False)
    for name, (a, b) in GROUPS.items():
        rel = np.linalg.norm(ge[a:b] - gx[a:b]) / np.linalg.norm(gx[a:b])
        assert rel < 3e-2, (name, rel)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * sign(g) up to eps
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)
