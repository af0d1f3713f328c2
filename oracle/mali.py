"""Float64 oracle of the multilevel accelerated lambda iteration (MALI) with
same-transition preconditioning and a diagonal approximate operator, the
population update Section 4.1 uses (after Rybicki & Hummer 1992), iterated until
the largest relative population change falls below a tolerance (Section 4.1:
1e-3).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU-baseline leg).

The atom, profiles, emissivities and collisional rates are those of
``oracle.atom``.  Per iteration, from the previous populations n':

* eta', chi' of every wavelength (Eqs. Eta/Chi plus the grey background) and
  the formal solution J' (any long-characteristics solver: plain or
  accelerated);
* the diagonal operator of the long-characteristics solve: a ray leaves its
  probe's own cell after l_k = 1 / (2 max(|d_x|, |d_z|)) cells, and that cell
  adds S (1 - e^{-chi l_k}) to I_k, so
      Lambda*_nu = sum_k w_k (1 - e^{-chi'_nu l_k})       (chi' per cell);
* same-transition preconditioning of line u -> l: the line's own emissivity
  enters J at the new populations through Lambda* with chi frozen at n', and
  the net radiative rate n_u A + n_u B_ul Jbar - n_l B_lu Jbar is linearised by
  taking the line opacity in front of Lambda* at n' too.  That gives the
  preconditioned rates
      R_ul = A_ul (1 - Psibar) + B_ul Jbar_eff,   R_lu = B_lu Jbar_eff,
      Psibar   = sum_nu w_nu phi_nu Lambda*_nu chi'_line,nu / chi'_nu,
      Jbar_eff = sum_nu w_nu phi_nu (J'_nu - Lambda*_nu eta'_line,nu / chi'_nu),
  (w_nu the line's frequency quadrature weights, phi_nu its profile), and the
  statistical equilibrium with these rates and the collisional ones is solved
  per cell for the MALI populations M(n').

The iteration is n <- M(n), as published (no damping or extrapolation).

Wavelength quadrature (a reading: the paper's atoms and grids are absent).  M
converges on the population workload only when each line's samples resolve its
profile at every temperature of the model.  With samples spanning +-4 Doppler
widths at 1e4 K, a 1e5 K cell sees only +-1.26 of its own Doppler widths: the
renormalised profile is flat across the samples, the cell is optically thick
per cell at every sampled frequency, 1 - Lambda* ~ e^{-chi l} is exponentially
small and exponentially sensitive to the previous populations, and M swings
such cells between far-apart states (measured on the 48 x 48 instance: the
largest relative change stays near 0.5 for 30 iterations).  With samples over
+-4 Doppler widths at 1e5 K the same iteration converges monotonically (the
largest change falls by ~0.82 per iteration; the Lambda iteration by ~0.99).
The MALI workload therefore samples the lines over +-4 Doppler widths at 1e5 K.
"""

from __future__ import annotations

import numpy as np

from . import atom as oa


def own_cell_lengths(dirs):
    """Path length (cells) from a cell centre to the cell boundary along each direction."""
    d = np.abs(np.asarray(dirs, dtype=np.float64).reshape(-1, 2))
    return 0.5 / d.max(axis=1)


def lambda_star(chi, dirs, weights):
    """Diagonal operator Lambda*[lambda][...] = sum_k w_k (1 - e^{-chi l_k})."""
    chi = np.asarray(chi, dtype=np.float64)
    ell = own_cell_lengths(dirs)
    w = np.asarray(weights, dtype=np.float64)
    out = np.zeros_like(chi)
    for lk, wk in zip(ell, w):
        out += wk * -np.expm1(-chi * lk)
    return out


def line_eta_chi(atom, lam_nm, tag, T, pops, cell_cm):
    """Line-only emissivity and opacity per cell [lambda][...] (0 at background samples)."""
    lam_nm = np.asarray(lam_nm, dtype=np.float64)
    nu = oa.C / (lam_nm * 1e-7)
    phi = oa.profiles(atom, lam_nm, tag, T)
    bs = oa.einstein_b(atom)
    eta = np.zeros((lam_nm.size,) + np.shape(T))
    chi = np.zeros_like(eta)
    for k in range(lam_nm.size):
        li = int(tag[k])
        if li < 0:
            continue
        lo, up, A, _ = atom["lines"][li]
        b_ul, b_lu = bs[li]
        f = oa.H * nu[k] / (4.0 * np.pi) * phi[k]
        eta[k] = f * pops[up] * A * cell_cm
        chi[k] = f * (pops[lo] * b_lu - pops[up] * b_ul) * cell_cm
    return eta, chi


def preconditioned(atom, lam_nm, tag, T, J, chi, eta_line, chi_line, lstar):
    """(Psibar, Jbar_eff) per line, shape [n_line][...]."""
    phi = oa.profiles(atom, lam_nm, tag, T)
    chi = np.asarray(chi, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(chi > 0, 1.0 / np.where(chi > 0, chi, 1.0), 0.0)
    psibar, jeff = [], []
    for li in range(len(atom["lines"])):
        w = oa.frequency_weights(lam_nm, tag, li)
        psibar.append(np.tensordot(w, phi * lstar * chi_line * inv, axes=1))
        jeff.append(np.tensordot(w, phi * (np.asarray(J, dtype=np.float64) - lstar * eta_line * inv), axes=1))
    return np.array(psibar), np.array(jeff)


def rate_matrix(atom, T, ne, psibar, jeff):
    """P[i][j][...]: preconditioned radiative plus collisional rates from level i to j."""
    zero = np.zeros((len(atom["lines"]),) + np.shape(T))
    P = oa.rate_matrix(atom, T, ne, zero)   # collisions and A_ul
    for li, ((lo, up, A, _), (b_ul, b_lu)) in enumerate(zip(atom["lines"], oa.einstein_b(atom))):
        P[lo, up] += b_lu * jeff[li]
        P[up, lo] += b_ul * jeff[li] - A * psibar[li]
    return P


def solve_populations(P, nh, live):
    """Statistical equilibrium of rate matrices P [nl][nl][cells] with sum n = n_H."""
    nl = P.shape[0]
    cells = P.shape[2]
    M = np.zeros((cells, nl, nl))
    for i in range(nl):
        for j in range(nl):
            if i != j:
                M[:, i, j] += P[j, i]
                M[:, i, i] -= P[i, j]
    M[:, 0, :] = 1.0
    rhs = np.zeros((cells, nl))
    rhs[:, 0] = np.asarray(nh, dtype=np.float64).reshape(-1)
    n = np.zeros((cells, nl))
    if live.any():
        n[live] = np.linalg.solve(M[live], rhs[live][..., None])[..., 0]
    return n.T


def mali_step(atom, lam_nm, tag, T, ne, nh, cell_cm, pops, J, dirs, weights):
    """M(pops): the MALI populations [nl][cells] from populations and their J (flat cell axis)."""
    T = np.asarray(T, dtype=np.float64).reshape(-1)
    ne = np.asarray(ne, dtype=np.float64).reshape(-1)
    eta, chi = oa.eta_chi(atom, lam_nm, tag, T, ne, pops, cell_cm)
    eta_l, chi_l = line_eta_chi(atom, lam_nm, tag, T, pops, cell_cm)
    lstar = lambda_star(chi, dirs, weights)
    psibar, jeff = preconditioned(atom, lam_nm, tag, T, J, chi, eta_l, chi_l, lstar)
    P = rate_matrix(atom, T, ne, psibar, jeff)
    return solve_populations(P, nh, T > 0)


def iterate(atom, lam_nm, tag, T, ne, nh, cell_cm, solve_J, dirs, weights, tol=1e-3, max_iter=200):
    """MALI from LTE until the largest relative change max |M(n) - n| / M(n) over
    non-empty cells and levels is below ``tol``.

    ``solve_J(eta, chi) -> J [lambda][cells]`` is the formal solver.  Returns
    ``(pops [nl][cells], n_iter, history of the largest relative changes)``;
    n_iter counts the MALI updates (formal solutions) performed."""
    T = np.asarray(T, dtype=np.float64).reshape(-1)
    ne = np.asarray(ne, dtype=np.float64).reshape(-1)
    nh = np.asarray(nh, dtype=np.float64).reshape(-1)
    live = T > 0
    pops = oa.lte_populations(atom, T, nh)
    hist = []
    for it in range(max_iter):
        eta, chi = oa.eta_chi(atom, lam_nm, tag, T, ne, pops, cell_cm)
        J = solve_J(eta, chi)
        new = mali_step(atom, lam_nm, tag, T, ne, nh, cell_cm, pops, J, dirs, weights)
        with np.errstate(invalid="ignore", divide="ignore"):
            change = np.where(live[None], np.abs(new - pops) / np.where(new > 0, new, 1.0), 0.0)
        hist.append(float(change.max()))
        pops = new
        if hist[-1] < tol:
            return pops, it + 1, hist
    return pops, max_iter, hist
