"""Pins of the Voigt oracle: closed forms of H(a, x), its normalisation and
asymptote, and the published accuracy of the HUM1WEI24 approximation against
the Faddeeva function."""

import math

import numpy as np
from scipy.special import erfcx

from oracle import voigt


def test_gaussian_and_centre_limits():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(voigt.voigt_h(0.0, x), np.exp(-x * x), rtol=1e-13, atol=1e-300)
    for a in (1e-3, 0.1, 1.0, 5.0):
        assert abs(voigt.voigt_h(a, 0.0) - erfcx(a)) < 1e-13 * erfcx(a)  # e^{a^2} erfc(a)


def test_normalisation_and_lorentz_wing():
    a = 0.05
    x = np.linspace(-2000, 2000, 4_000_001)
    H = voigt.voigt_h(a, x)
    assert abs(np.trapezoid(H, x) / math.sqrt(math.pi) - 1) < 2e-4   # wings beyond 2000 lost
    xw = 300.0
    assert abs(voigt.voigt_h(a, xw) / (a / (math.sqrt(math.pi) * xw * xw)) - 1) < 1e-4


def test_weideman_coefficients_reproduce_w():
    # Weideman's expansion alone (without Humlicek's region) converges to w in the
    # upper half plane: with 24 terms the error is small near the line centre.
    L, a = voigt.weideman_coefficients(24)
    assert abs(L - math.sqrt(24 / math.sqrt(2))) < 1e-15 and a.size == 24
    x = np.linspace(-5, 5, 101)
    for y in (0.01, 0.3, 2.0):
        ref = voigt.voigt_h(y, x)
        approx = voigt.voigt_h(y, x, method="hum1wei24")
        assert np.max(np.abs(approx - ref) / ref) < 5e-5


def test_hum1wei24_accuracy_over_the_line():
    # relative accuracy over |x| <= 100, a in [1e-3, 1e-1] (the damping range of the
    # dynamic workload); Schreier (2018) reports ~1e-4 or better for this combination
    x = np.concatenate([np.linspace(-30, 30, 6001), np.geomspace(30, 100, 200)])
    worst = 0.0
    for a in np.geomspace(1e-3, 1e-1, 9):
        ref = voigt.voigt_h(a, x)
        approx = voigt.voigt_h(a, x, method="hum1wei24")
        worst = max(worst, float(np.max(np.abs(approx - ref) / ref)))
    assert worst < 1e-4, worst


def test_hum1wei24_error_by_region():
    # where HUM1WEI24's error sits: Humlicek's region I (|x| + a >= 15, an
    # asymptotic form whose next term is ~1/(2 z^4)) up to 5.2e-5 at its edge;
    # Weideman's 24-term sum below it within 3e-6 over the workload's damping range
    x = np.concatenate([np.linspace(-30, 30, 60001), np.geomspace(30, 2000, 2000)])
    for a in np.geomspace(1e-3, 1e-1, 5):
        ref = voigt.voigt_h(a, x)
        err = np.abs(voigt.voigt_h(a, x, method="hum1wei24") - ref) / ref
        s = np.abs(x) + a
        assert err[s < 15].max() < 3e-6, (a, err[s < 15].max())
        assert err[s >= 15].max() < 5.2e-5, (a, err[s >= 15].max())
