"""Spectral bounds, normalisation, flip, validity and model choice
(TEST INFRASTRUCTURE ONLY).

Follows Sec. III A (Eqs. H', mu', beta', rescaling, H0, conditions), Sec. IV C
(Eq. flip) and the Appendix A program, in that order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def gershgorin(H: np.ndarray):
    """Appendix A: e_min = min_i(H_ii - R_i), e_max = max_i(H_ii + R_i),
    R_i = sum_{j != i} |H_ij|."""
    H = np.asarray(H, dtype=np.float64)
    d = np.diag(H)
    R = np.sum(np.abs(H), axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def gershgorin_loops(H):
    """The same bounds with explicit loops (tiny matrices; brute-force pin)."""
    n = len(H)
    lo, hi = math.inf, -math.inf
    for i in range(n):
        r = 0.0
        for j in range(n):
            if j != i:
                r += abs(H[i][j])
        lo = min(lo, H[i][i] - r)
        hi = max(hi, H[i][i] + r)
    return lo, hi


def normalise(e_min: float, e_max: float, mu: float, beta: float):
    """Eqs. mu' and beta': mu' = (e_max - mu)/(e_max - e_min),
    beta' = (e_max - e_min) beta.  (Alg. 2 prints beta' = (e_max - e_min) beta';
    the right-hand beta' is read as beta, as in Eq. beta' and Appendix A.)"""
    W = e_max - e_min
    return (e_max - mu) / W, W * beta


def flip_needed(mu_p: float) -> bool:
    """Eq. flip is used when mu' > 1/2 (strict, as in Appendix A)."""
    return mu_p > 0.5


def is_valid(mu_p: float, beta_p: float, beta0: float, mu0: float) -> bool:
    """Region of validity: the spectrum of H0 lies in [0, 1], i.e.
    0 <= (beta'/beta0)(0 - mu') + mu0 and (beta'/beta0)(1 - mu') + mu0 <= 1
    (the inequalities stated just before Eq. conditions).  This linear form
    equals Eq. conditions for 0 < mu' < 1 and stays defined when mu lies
    outside [e_min, e_max] (reading for mu' outside (0, 1))."""
    s = beta_p / beta0
    return (s * (0.0 - mu_p) + mu0 >= 0.0) and (s * (1.0 - mu_p) + mu0 <= 1.0)


def beta_max(mu_p: float, beta0: float, mu0: float) -> float:
    """Largest valid beta' for this mu' (Appendix A: min(mu0/mu', (1-mu0)/(1-mu'))
    beta0), each branch only where its denominator is positive."""
    cands = []
    if mu_p > 0:
        cands.append(mu0 / mu_p)
    if mu_p < 1:
        cands.append((1.0 - mu0) / (1.0 - mu_p))
    return beta0 * min(cands) if cands else math.inf


@dataclass
class Table:
    """One model of the model set (Sec. III A 2, "a set of models")."""
    theta: tuple
    beta0: float
    mu0: float
    alpha: float = 0.842704
    theta_entropy: tuple | None = None   # None: reuse theta (theta_fermi strategy)
    name: str = ""

    @property
    def L(self):
        return len(self.theta)


def select_model(tables, mu_p: float, beta_p: float, min_layers: bool = False):
    """Workflow step 4: a model whose region of validity contains (beta', mu').
    Reading (the paper only asks for one that contains it, and names the
    minimum layer count as one favourable property): by default the valid
    model with the smallest beta0 (least amplified rounding), ties broken by
    fewer layers; with ``min_layers`` the valid model with the fewest layers,
    ties broken by the smaller beta0.  Then by position in the set.  Returns the
    index or -1."""
    def key(t):
        return (t.L, t.beta0) if min_layers else (t.beta0, t.L)
    best = -1
    for k, t in enumerate(tables):
        if not is_valid(mu_p, beta_p, t.beta0, t.mu0):
            continue
        if best < 0 or key(t) < key(tables[best]):
            best = k
    return best


@dataclass
class RescaleRecord:
    e_min: float
    e_max: float
    mu_p: float          # after the flip
    beta_p: float        # after clamping (if any)
    flip: bool
    model: int
    valid: bool


def rescale(H: np.ndarray, mu: float, kT: float, tables, clamp: bool = False, lanczos: bool = False,
            min_layers: bool = False):
    """Bounds -> (H', mu', beta') -> flip -> model -> H0 (Sec. III A, Appendix A).

    Returns (H0, record).  With ``clamp`` the paper's behaviour outside the
    region of validity is reproduced (beta' lowered to the largest valid value of
    the largest-beta0 model); otherwise the record says ``valid=False`` and H0 is
    None.  Degenerate spectrum (e_max == e_min, only H = cI): the normalisation
    divides by zero, so the equivalent form H0 = mu0 I + (beta/beta0)(mu I - H)
    is used with no flip (reading; the two agree whenever both are defined).
    With ``lanczos`` the bounds are those of ``oracle.lanczos.bounds`` (the
    Gershgorin interval tightened by a few Lanczos steps) instead; ``min_layers``
    selects the model policy of ``select_model``."""
    beta = 1.0 / kT
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    I = np.eye(n)
    if lanczos:
        from . import lanczos as lz
        e_min, e_max = lz.bounds(H)
    else:
        e_min, e_max = gershgorin(H)
    if e_max == e_min:
        best = -1
        def key(t):
            return (t.L, t.beta0) if min_layers else (t.beta0, t.L)
        for k, t in enumerate(tables):
            x = t.mu0 + (beta / t.beta0) * (mu - e_min)
            if 0.0 <= x <= 1.0 and (best < 0 or key(t) < key(tables[best])):
                best = k
        rec = RescaleRecord(e_min, e_max, math.nan, 0.0, False, best, best >= 0)
        if best < 0:
            return None, rec
        t = tables[best]
        return t.mu0 * I + (beta / t.beta0) * (mu * I - H), rec
    W = e_max - e_min
    H_p = (e_max * I - H) / W                        # Eq. H'
    mu_p, beta_p = normalise(e_min, e_max, mu, beta)  # Eqs. mu', beta'
    flip = flip_needed(mu_p)
    if flip:                                          # Eq. flip
        H_p = I - H_p
        mu_p = 1.0 - mu_p
    k = select_model(tables, mu_p, beta_p, min_layers=min_layers)
    valid = k >= 0
    if not valid:
        if not clamp:
            return None, RescaleRecord(e_min, e_max, mu_p, beta_p, flip, -1, False)
        k = max(range(len(tables)), key=lambda j: tables[j].beta0)
        beta_p = min(beta_p, beta_max(mu_p, tables[k].beta0, tables[k].mu0))
    t = tables[k]
    H0 = (beta_p / t.beta0) * (H_p - mu_p * I) + t.mu0 * I   # Eq. H0
    return H0, RescaleRecord(e_min, e_max, mu_p, beta_p, flip, k, valid)


def x0_of_eigenvalue(eps, mu: float, kT: float, rec: RescaleRecord, table: Table):
    """Image of an eigenvalue eps of H under the map H -> H0 of ``rescale``
    (Eq. H0 applied to the eigenvalue (e_max - eps)/W of H', flipped if needed)."""
    eps = np.asarray(eps, dtype=np.float64)
    if rec.e_max == rec.e_min:
        return table.mu0 + (1.0 / kT / table.beta0) * (mu - eps)
    W = rec.e_max - rec.e_min
    xp = (rec.e_max - eps) / W
    if rec.flip:
        xp = 1.0 - xp
    return (rec.beta_p / table.beta0) * (xp - rec.mu_p) + table.mu0
