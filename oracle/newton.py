"""Chemical potential for a prescribed electron count (Sec. III A 4): Newton-
Raphson on g(mu) = N_occ - Tr D(mu) (Eq. g)  (TEST INFRASTRUCTURE ONLY).

The derivative comes from the logistic dependence of D on mu.  Differentiating
the Fermi operator D = [exp(beta (H - mu I)) + I]^-1 (Eq. FD_Func) gives
dD/dmu = +beta D (I - D); the printed Eq. drho carries the opposite sign, which
would send each step away from the root.  With the sign of the definition
(reading taken here):

    g'(mu) = -Tr(dD/dmu) = -beta (Tr D - Tr D^2)               (Eq. dg, sign fixed)
    Delta mu = -g / g' = (N_occ - Tr D) / (beta (Tr D - Tr D^2))   (Eq. delta_mu, sign fixed)

with Tr D^2 = ||D||_F^2 for symmetric D (Eq. tr(D^2)), i.e. no extra matrix
product.  Every step re-evaluates D at the new mu with the whole method
(bounds, rescale, flip, model choice, the recursion), here through
``pipeline.method_exact`` (the method's exact result on the eigenvalues).

Readings where the paper is silent:
* a step is limited to |Delta mu| <= W / 16, W = e_max - e_min the Gershgorin
  width (far from the root, with mu in a gap of the spectrum, Tr(D - D^2) is
  tiny and the raw step overshoots the spectrum);
* once |g| <= tol the instance is left unchanged;
* a step is skipped when Tr D - Tr D^2 <= 0 (D idempotent to rounding) or when
  the instance is outside every model's region of validity.
"""
from __future__ import annotations

import numpy as np

from . import pipeline, rescale

STEP_CAP = 1.0 / 16.0          # |Delta mu| <= STEP_CAP * W


def newton_step(n_occ: float, trD: float, trD2: float, kT: float, width: float, tol: float):
    """Delta mu of one step (0 when converged or when the step is undefined)."""
    g = n_occ - trD
    if abs(g) <= tol:
        return 0.0
    gp = (trD - trD2) / kT                     # -g'(mu) = beta Tr(D - D^2)
    if not gp > 0.0:
        return 0.0
    cap = STEP_CAP * width
    return float(np.clip(g / gp, -cap, cap))


def newton_mu(H: np.ndarray, n_occ: float, mu: float, kT: float, tables, iterations: int, tol: float):
    """``iterations`` Newton updates from the initial guess mu.  Returns
    (final mu, history of (mu, Tr D, Tr D^2, Delta mu) per update, the
    method-exact result at the final mu)."""
    hist = []
    for _ in range(iterations):
        r = pipeline.method_exact(H, mu, kT, tables)
        if r["D"] is None:
            break
        rec = r["rec"]
        d = newton_step(n_occ, r["trD"], r["frobD"], kT, rec.e_max - rec.e_min, tol)
        hist.append((mu, r["trD"], r["frobD"], d))
        mu = mu + d
    return mu, hist, pipeline.method_exact(H, mu, kT, tables)


def method_electron_count(H: np.ndarray, mu: float, kT: float, tables) -> float:
    """Tr D_rec(mu): the electron count the method gives at mu."""
    r = pipeline.method_exact(H, mu, kT, tables)
    return r["trD"]


def method_mu_bisection(H: np.ndarray, n_occ: float, kT: float, tables, lo: float, hi: float,
                        iters: int = 100) -> float:
    """The root of Tr D_rec(mu) = n_occ by bisection on [lo, hi] (Tr D_rec is
    increasing in mu); an independent route to the root Newton converges to."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if method_electron_count(H, mid, kT, tables) > n_occ:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def gershgorin_width(H: np.ndarray) -> float:
    lo, hi = rescale.gershgorin(H)
    return hi - lo
