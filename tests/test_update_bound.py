"""Accuracy of the per-segment factor 1 - e^{-tau} as the solvers evaluate it.

The kernels take g = min(P5(tau), (1 + 2^-21) - e), with P5 the degree-5 Taylor
polynomial of 1 - e^{-tau} (Horner in x = -tau log2(e), float32 coefficients
from ln 2) and e = 2^x from the special-function unit.  The argument is:
P5 >= 1 - e^{-tau} for tau >= 0 (alternating series, negative Lagrange
remainder), and (1 + 2^-21) - e >= 1 - e^{-tau} as long as e exceeds 2^x by
less than 2^-21, so the minimum of the two upper bounds is close to exact.
This test evaluates the same float32 arithmetic on the CPU with e off by up to
8 x 2^-24 below and 7 x 2^-24 above its exact value (near 1; a few ulps
elsewhere), checks the relative error bound against float64 expm1, and that a
mistake in the construction (a dropped series term, no 2^-21 margin) breaks
it.  The GPU parity tests (1e-5 against the float64 oracle, with many thin
segments) check the same on the hardware.
"""

import numpy as np

LN2 = np.log(2.0)
LOG2E = 1.0 / LN2


def coefs(n=5):
    # -(ln 2)^k / k!, k = 1..n, rounded to float32 (the kernel's constants)
    c, out = 1.0, []
    for k in range(1, n + 1):
        c *= LN2 / k
        out.append(np.float32(-c))
    return out


def series_x_p(x, n=5):
    """x * p(x) in float32 Horner form, p = sum_k c_k x^(k-1)."""
    c = coefs(n)
    p = np.full_like(x, c[-1])
    for ck in reversed(c[:-1]):
        p = (x * p + ck).astype(np.float32)
    return (x * p).astype(np.float32)


def factor(tau, ulps, margin=2.0 ** -21, n=5):
    """g as the kernels form it, with the 2^x result off by `ulps` units of 2^-24
    (the float32 spacing just below 1) for results in [0.5, 1], and by `ulps`
    float32 ulps of the result below 0.5."""
    x = (np.float32(-LOG2E) * tau.astype(np.float32)).astype(np.float32)
    e_true = np.exp2(x.astype(np.float64))
    unit = np.where(e_true >= 0.5, 2.0 ** -24, np.spacing(e_true.astype(np.float32)).astype(np.float64))
    e = (e_true + ulps * unit).astype(np.float32)
    one_plus = np.float32(1.0 + margin)
    g = np.minimum(series_x_p(x, n), (one_plus - e).astype(np.float32))
    exact = -np.expm1(x.astype(np.float64) * LN2)
    return g.astype(np.float64), exact


TAU = np.concatenate([np.logspace(-8, 2.5, 120001), np.linspace(0.05, 0.5, 90001)])


def test_relative_error_bound_with_sfu_error_below_2_to_minus_21():
    worst = 0.0
    for ulps in (-8, -4, -1, 0, 1, 4, 7):
        g, exact = factor(TAU, ulps)
        rel = np.abs(g - exact) / exact
        worst = max(worst, float(rel.max()))
        if ulps == 0:
            assert rel.max() < 2.3e-6  # exact 2^x: the crossover near tau = 0.27
    assert worst < 4.0e-6, worst


def test_small_tau_uses_the_series():
    # below tau ~ 0.1 the result is the series, accurate to float32 rounding
    tau = np.logspace(-8, -1, 20001)
    for ulps in (-8, 0, 7):
        g, exact = factor(tau, ulps)
        assert (np.abs(g - exact) / exact).max() < 3e-7


def test_zero_and_opaque_limits():
    g, _ = factor(np.array([0.0]), 0)
    assert g[0] == 0.0
    g, exact = factor(np.array([50.0, 300.0]), 0)
    assert np.all(np.abs(g - 1.0) < 1e-6) and np.all(exact == 1.0)


def test_planted_mistakes_break_the_bound():
    # a dropped series term or a missing margin must be caught by the bound above
    g, exact = factor(TAU, 0, n=4)
    assert (np.abs(g - exact) / exact).max() > 4.0e-6
    g, exact = factor(TAU, 4, margin=0.0)
    assert (np.abs(g - exact) / exact).max() > 4.0e-6
