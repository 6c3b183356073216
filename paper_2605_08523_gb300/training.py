"""Host-side preparation for coefficient training (a7; Sec. II C): the fixed
sample set, the initial table, and a driver around ftsp2_train_coeffs.

The fit itself (residuals, reverse-mode Jacobian, J^T J, J^T r, the damped
normal equations and geodesic acceleration) runs in the library; this module
only builds inputs and collects outputs.

* Samples: a deterministic quantile grid of the density p(x) ~ 1 + |f'(x)| on
  [0, 1] (Sec. II C 1: sampling that follows the derivative of the Fermi
  function targets the maximum error; the set is fixed for the whole fit).
* Initial table: the SP2 sequence for a known chemical potential (Eq. sp2-mu)
  at mu0, embedded in MLSP2 form (Appendix C: X^2 -> (1, 0, 0, 0),
  2X - X^2 -> (-1, 2, 0, 0)), with an affine contraction of the input about
  mu0 folded into layer 0 so that the slope at mu0 equals beta0 / 4 (the
  slope of the target logistic).
"""
from __future__ import annotations

import math

import numpy as np


def _logistic(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    pos = t >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-t[pos]))
    e = np.exp(t[~pos])
    out[~pos] = e / (1.0 + e)
    return out


def sample_points(N: int, beta0: float, mu0: float, weighting: str = "derivative", fine: int = 2_000_001):
    """N points on [0, 1] at the quantiles (i + 1/2)/N of p(x), with
    p ~ 1 + |f'| ("derivative"), sqrt(1 + f'^2) ("arclength") or 1
    ("uniform"), f(x) = 1/(1 + exp(-beta0 (x - mu0)))."""
    g = np.linspace(0.0, 1.0, fine)
    if weighting == "uniform":
        p = np.ones_like(g)
    else:
        f = _logistic(beta0 * (g - mu0))
        fp = beta0 * f * (1.0 - f)
        p = 1.0 + fp if weighting == "derivative" else np.sqrt(1.0 + fp * fp)
    cdf = np.zeros_like(g)
    cdf[1:] = np.cumsum(0.5 * (p[1:] + p[:-1]) * (g[1] - g[0]))
    cdf /= cdf[-1]
    return np.interp((np.arange(N) + 0.5) / N, cdf, g)


def sp2_sequence(mu_p: float, L: int):
    """Branch choices of Eq. sp2-mu: +1 for X^2 when |m^2 - mu'| < |2m - m^2 - mu'|,
    else -1 for 2X - X^2; m follows the chosen polynomial from m = mu'."""
    m, out = mu_p, []
    for _ in range(L):
        sq, up = m * m, 2.0 * m - m * m
        if abs(sq - mu_p) < abs(up - mu_p):
            out.append(1)
            m = sq
        else:
            out.append(-1)
            m = up
    return out


def sp2_init(L: int, beta0: float, mu0: float):
    """(L, 4) initial table (see module docstring)."""
    sig = sp2_sequence(mu0, L)
    th = np.array([(1.0, 0.0, 0.0, 0.0) if s > 0 else (-1.0, 2.0, 0.0, 0.0) for s in sig])
    # slope of the composition at mu0: product of p_i'(m_i) along the trajectory
    m, slope = mu0, 1.0
    for a, b, c, _ in th:
        slope *= 2.0 * a * m + b
        m = a * m * m + b * m + c
    kappa = min(1.0, (beta0 / 4.0) / slope) if slope > 0 else 1.0
    shift = mu0 * (1.0 - kappa)
    a, b, c, d = th[0]
    th[0] = (a * kappa * kappa, 2.0 * a * kappa * shift + b * kappa, a * shift * shift + b * shift + c, d)
    return th


def sp2_alt_init(L: int, mu0: float):
    """(L + 1, 2) table of the one-term form (Eq. mlsp2_alt) computing the SP2
    sequence at mu0 exactly: the state y is x or 1 - x, and both branches are
    squares, X^2 = (0 + y)^2 and 1 - (2X - X^2) = (-1 + y)^2 (or the same with
    the roles of the offsets swapped when y = 1 - x); the output row undoes a
    final y = 1 - x."""
    alt = np.zeros((L + 1, 2))
    flipped = False
    for i, s in enumerate(sp2_sequence(mu0, L)):
        if s > 0:
            alt[i, 0] = -1.0 if flipped else 0.0
            flipped = False
        else:
            alt[i, 0] = 0.0 if flipped else -1.0
            flipped = True
    alt[L] = (1.0, -1.0) if flipped else (0.0, 1.0)
    return alt


def skip_from_mlsp2(theta):
    """(L + 1, 4) Skip-SP2 table (one stored layer, one accumulator, no
    accumulator feedback) computing the same function as Eq. mlsp2 rows theta
    (the Appendix embedding): each quadratic is a_i (x + b_i / (2 a_i))^2 + e_i
    with e_i = c_i - b_i^2 / (4 a_i); the square is the next layer's x~, whose
    combination carries a_{i-1} and e_{i-1}; the accumulator weights pick up
    a_{i-1}, and the constants e collect in A_0."""
    th = np.asarray(theta, dtype=np.float64)
    L = th.shape[0]
    a, b, c, d = th[:, 0], th[:, 1], th[:, 2], th[:, 3]
    e = c - b * b / (4.0 * a)
    tab = np.zeros((L + 1, 4))
    tab[0] = (b[0] / (2.0 * a[0]), 1.0, 0.0, d[0])
    for i in range(1, L):
        tab[i] = (e[i - 1] + b[i] / (2.0 * a[i]), a[i - 1], 0.0, d[i] * a[i - 1])
    tab[L, 0] = e[L - 1] + float(np.dot(d[1:], e[:-1]))
    tab[L, 1] = a[L - 1]
    return tab


def train_skip_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                     nsamples: int = 100_000, skip_init=None, accel: bool = True, device="cuda"):
    """Fit a Skip-SP2 table on the GPU (ftsp2_train_coeffs_skip); the default
    start is the embedding of the SP2 initial guess."""
    import torch
    x = torch.from_numpy(sample_points(nsamples, beta0, mu0)).to(device)
    t0 = skip_from_mlsp2(sp2_init(L, beta0, mu0)) if skip_init is None else np.asarray(skip_init, dtype=np.float64)
    return ft.ftsp2_train_coeffs_skip(target, beta0, mu0, t0, x, iterations=iterations, accel=accel, alpha=alpha)


def train_alt_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                    nsamples: int = 100_000, alt_init=None, accel: bool = True, device="cuda"):
    """Fit a table of the one-term form on the GPU (ftsp2_train_coeffs_alt)."""
    import torch
    x = torch.from_numpy(sample_points(nsamples, beta0, mu0)).to(device)
    a0 = sp2_alt_init(L, mu0) if alt_init is None else np.asarray(alt_init, dtype=np.float64)
    return ft.ftsp2_train_coeffs_alt(target, beta0, mu0, a0, x, iterations=iterations, accel=accel, alpha=alpha)


def train_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                nsamples: int = 100_000, theta_init=None, accel: bool = True, device="cuda"):
    """Fit a table on the GPU (ftsp2_train_coeffs).  Returns (theta, report)."""
    import torch
    x = torch.from_numpy(sample_points(nsamples, beta0, mu0)).to(device)
    th0 = sp2_init(L, beta0, mu0) if theta_init is None else np.asarray(theta_init, dtype=np.float64)
    return ft.ftsp2_train_coeffs(target, beta0, mu0, th0, x, iterations=iterations, accel=accel, alpha=alpha)


def layer_count(beta_p: float) -> float:
    """Eq. layer count: n_l = ln(beta'/4) / ln(2 phi), phi = 1/varphi."""
    phi = 2.0 / (1.0 + math.sqrt(5.0))
    return math.log(beta_p / 4.0) / math.log(2.0 * phi)
