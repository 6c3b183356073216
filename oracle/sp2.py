"""SP2 with a known chemical potential, its MLSP2 embedding and the layer-count
estimate (TEST INFRASTRUCTURE ONLY).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0    # varphi
PHI = 1.0 / GOLDEN                        # phi = varphi^-1 (Sec. IV B)


def sp2_mu_sequence(mu_p: float, L: int):
    """Eq. sp2-mu: starting from mu_0 = mu', layer i applies X^2 when
    |mu_i^2 - mu'| < |2 mu_i - mu_i^2 - mu'| and 2X - X^2 otherwise, and
    mu_{i+1} is the image of mu_i under the chosen polynomial.  Returns the
    list of sigma_i (+1 for X^2, -1 for 2X - X^2) and the final mu_n."""
    sig = []
    m = mu_p
    for _ in range(L):
        sq, up = m * m, 2.0 * m - m * m
        if abs(sq - mu_p) < abs(up - mu_p):
            sig.append(+1)
            m = sq
        else:
            sig.append(-1)
            m = up
    return sig, m


def sp2_table(mu_p: float, L: int):
    """MLSP2 coefficients of the SP2 sequence (Appendix C, SP2 in MLSP2):
    sigma = +1 -> (1, 0, 0, 0), sigma = -1 -> (-1, 2, 0, 0); no accumulator.
    (Appendix C prints the second distance as |2 mu_i^2 - mu_i^2 - mu'|; read as
    |2 mu_i - mu_i^2 - mu'| to agree with Eq. sp2-mu.)"""
    sig, _ = sp2_mu_sequence(mu_p, L)
    return tuple((1.0, 0.0, 0.0, 0.0) if s > 0 else (-1.0, 2.0, 0.0, 0.0) for s in sig)


def layer_count(beta_p: float) -> float:
    """Eq. layer count: n_l = ln(beta'/4) / ln(2 varphi^-1)."""
    return math.log(beta_p / 4.0) / math.log(2.0 * PHI)


def beta0_for_layers(n_l: float) -> float:
    """Sec. IV C: beta0 = 4 (2 phi)^n_l."""
    return 4.0 * (2.0 * PHI) ** n_l


def f0(x):
    return x * x


def f1(x):
    return 2.0 * x - x * x


def alternating_composition(x, n_l: int):
    """f_{n_l mod 2} o ... o f_1 o f_0 applied to x (Sec. IV B)."""
    y = np.asarray(x, dtype=np.float64)
    for i in range(n_l):
        y = f0(y) if i % 2 == 0 else f1(y)
    return y


def slope_at(theta, x: float, h: float = 1e-7) -> float:
    """Central-difference slope of the scalar MLSP2 output at x."""
    from .mlsp2 import mlsp2_scalar
    return float((mlsp2_scalar([x + h], theta)[0] - mlsp2_scalar([x - h], theta)[0]) / (2 * h))
