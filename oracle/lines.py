"""Float64 oracle for the MIP-0 emissivity and opacity of a static continuum + line model.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

Section 2, Eqs. EtaTot and ChiTot: eta = sum_l eta_l + eta_bg and
chi = sum_l chi_l + chi_bg.  For the static synthetic model the background is
a continuum with opacity chi_c and source function S_c, and the single line
has opacity chi_l(lambda) = ratio * chi_c * exp(-(dlam / dld)^2) (a Gaussian
profile normalised to its peak, so ``ratio`` is the peak line-to-continuum
opacity ratio) and source function S_l; eta_x = chi_x * S_x for each part.
"""

from __future__ import annotations

import numpy as np


def line_eta_chi(chi_c, s_c, s_l, ratio, dld, dlam):
    """Return float64 ``(eta, chi)`` of shape ``[n_lambda][nz][nx]``."""
    chi_c = np.asarray(chi_c, dtype=np.float64)
    s_c = np.asarray(s_c, dtype=np.float64)
    s_l = np.asarray(s_l, dtype=np.float64)
    ratio = np.asarray(ratio, dtype=np.float64)
    dld = np.asarray(dld, dtype=np.float64)
    dlam = np.asarray(dlam, dtype=np.float64)
    L = dlam.size
    eta = np.empty((L,) + chi_c.shape)
    chi = np.empty((L,) + chi_c.shape)
    for l in range(L):
        chi_l = ratio * chi_c * np.exp(-(dlam[l] / dld) ** 2)
        chi[l] = chi_c + chi_l
        eta[l] = chi_c * s_c + chi_l * s_l
    return eta, chi
