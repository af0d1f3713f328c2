"""Float64 oracle of the Voigt function H(a, x) = Re w(x + i a).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

* ``exact``: the Faddeeva function from scipy (``scipy.special.wofz``): the accuracy reference.
* ``hum1wei24``: the approximation Section 3.2 names (Schreier 2018, "HUM1WEI24"),
  restated from its published sources, in float64 (``method="hum1wei24"``):
    - |x| + y >= 15: region I of Humlicek (1982), w(z) = i z / (sqrt(pi) (z^2 - 1/2));
    - otherwise Weideman (1994) with N = 24 terms:
        w(z) = 2 p(Z) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
        Z = (L + i z) / (L - i z),  p(Z) = sum_{n=1..N} a_n Z^(n-1),  L = sqrt(N / sqrt 2),
      where a_n are the Fourier coefficients of f(theta) = exp(-t^2) (L^2 + t^2),
      t = L tan(theta / 2), by the trapezoid rule on 2M = 4N points (f(-pi) = 0).
The GPU evaluates the same function H in float32 by its own scheme (its
header states it); parity tests bound that scheme against ``exact`` and use
``hum1wei24`` (the method's form, branch taken in float64) as the oracle of
the moving-medium solves.
"""

from __future__ import annotations

import numpy as np
from scipy.special import wofz

N_TERMS = 24


def weideman_coefficients(n: int = N_TERMS):
    """(L, a[1..n]) of Weideman's rational expansion, from the definition."""
    M = 2 * n
    L = np.sqrt(n / np.sqrt(2.0))
    k = np.arange(-M + 1, M)                 # theta = -pi (k = -M) contributes f = 0
    theta = k * np.pi / M
    t = L * np.tan(theta / 2.0)
    f = np.exp(-t * t) * (L * L + t * t)
    a = np.array([np.sum(f * np.cos(m * theta)) / (2 * M) for m in range(1, n + 1)])
    return L, a


_L, _A = weideman_coefficients()


def hum1wei24(x, y):
    """Complex w(x + i y) by HUM1WEI24 (y >= 0), float64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = x + 1j * y
    s = np.abs(x) + y
    out = np.empty(np.broadcast(x, y).shape, dtype=np.complex128)
    far = s >= 15.0
    with np.errstate(divide="ignore", invalid="ignore"):
        zf = np.broadcast_to(z, out.shape)[far]
        out[far] = 1j * zf / (np.sqrt(np.pi) * (zf * zf - 0.5))
        zn = np.broadcast_to(z, out.shape)[~far]
        den = _L - 1j * zn
        Z = (_L + 1j * zn) / den
        p = np.zeros_like(Z)
        for a in _A[::-1]:                    # Horner, highest power first
            p = p * Z + a
        out[~far] = 2.0 * p / (den * den) + 1.0 / (np.sqrt(np.pi) * den)
    return out


def voigt_h(a, x, method: str = "exact"):
    """H(a, x) = Re w(x + i a) (a >= 0)."""
    if method == "exact":
        return np.real(wofz(np.asarray(x, dtype=np.float64) + 1j * np.asarray(a, dtype=np.float64)))
    if method == "hum1wei24":
        return np.real(hum1wei24(x, a))
    raise ValueError(method)
