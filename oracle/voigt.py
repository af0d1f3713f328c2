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
* ``hum1wei24_cf``: the form the GPU evaluates: the same, except that for
  5 <= |x| + y < 15 the Weideman sum is replaced by the 8-term Laplace continued
  fraction w(z) = (i / sqrt(pi)) / (z - (1/2) / (z - 1 / (z - (3/2) / ...)))
  (Gautschi 1970), evaluated from the innermost term.  In float32 the Weideman
  sum cancels O(1) terms down to H ~ 1e-5 in the line wings; the continued
  fraction does not.
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


def laplace_cf(x, y, n_terms: int = 8):
    """w(x + i y) from the Laplace continued fraction with ``n_terms`` levels."""
    z = np.asarray(x, dtype=np.float64) + 1j * np.asarray(y, dtype=np.float64)
    f = z.copy()
    for k in range(n_terms, 0, -1):
        f = z - (k / 2.0) / f
    return 1j / (np.sqrt(np.pi) * f)


def hum1wei24_cf(x, y):
    """w(x + i y): Humlicek region I for s >= 15, continued fraction for 5 <= s < 15,
    Weideman-24 for s < 5 (s = |x| + y).  The branch is chosen with s computed in
    float32, the precision in which the GPU kernel takes the same decision; the
    values are float64."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x, y = np.broadcast_arrays(x, y)
    s32 = np.abs(x).astype(np.float32) + y.astype(np.float32)
    z = x + 1j * y
    out = np.empty(x.shape, dtype=np.complex128)
    far = s32 >= np.float32(15.0)
    band = (s32 >= np.float32(5.0)) & ~far
    near = ~(far | band)
    with np.errstate(divide="ignore", invalid="ignore"):
        out[far] = 1j * z[far] / (np.sqrt(np.pi) * (z[far] * z[far] - 0.5))
    out[band] = laplace_cf(x[band], y[band])
    out[near] = hum1wei24(x[near], y[near])   # s < 5 < 15: the Weideman branch
    return out


def voigt_h(a, x, method: str = "exact"):
    """H(a, x) = Re w(x + i a) (a >= 0)."""
    if method == "exact":
        return np.real(wofz(np.asarray(x, dtype=np.float64) + 1j * np.asarray(a, dtype=np.float64)))
    if method == "hum1wei24":
        return np.real(hum1wei24(x, a))
    if method == "hum1wei24_cf":
        return np.real(hum1wei24_cf(x, a))
    raise ValueError(method)
