"""Training the per-layer coefficients (TEST INFRASTRUCTURE ONLY).

Sec. II C: the model is fitted on scalar samples x in [0, 1] (eigenvalues of a
normalised Hamiltonian) drawn once from a fixed density and never re-sampled;
the fit is nonlinear least squares by Levenberg-Marquardt, optionally with
geodesic acceleration.

Readings (the paper names the methods but gives no values):
* samples: a deterministic quantile grid of p(x) ~ 1 + |f'(x)| (or uniform, or
  arc length sqrt(1 + f'^2)), x_s = F^-1((s + 1/2)/N) with F the CDF of p;
* Fermi target in the model frame: 1/(1 + exp(-beta0 (x - mu0))) (the
  increasing logistic that the printed weights approximate); entropy target:
  s(beta0 (x - mu0)) of Eq. entropy;
* LM: solve (J^T J + lambda diag(J^T J)) v = -J^T r; accept when the cost
  drops, then lambda /= 10, else lambda *= 10 (Marquardt's scaling and
  update);
* geodesic acceleration: r_vv = (2/h)((r(theta + h v) - r(theta))/h - J v),
  a = -(J^T J + lambda diag(J^T J))^-1 J^T r_vv, step v + a/2, taken only if
  2 |a| / |v| <= 0.75 (the acceptance rule of Transtrum and Sethna's
  geodesic-acceleration LM, written from its published description).
"""
from __future__ import annotations

import math

import numpy as np

from . import fermi

LN2 = math.log(2.0)


def fermi_target(x, beta0: float, mu0: float):
    return fermi.fermi(-np.asarray(x, dtype=np.float64), -mu0, 1.0 / beta0)


def entropy_target(x, beta0: float, mu0: float):
    return fermi.entropy_of_t(beta0 * (np.asarray(x, dtype=np.float64) - mu0))


def _density(x, beta0, mu0, weighting):
    if weighting == "uniform":
        return np.ones_like(x)
    f = fermi_target(x, beta0, mu0)
    fp = beta0 * f * (1.0 - f)
    if weighting == "derivative":
        return 1.0 + np.abs(fp)
    if weighting == "arclength":
        return np.sqrt(1.0 + fp * fp)
    raise ValueError(weighting)


def sample_grid(N: int, beta0: float, mu0: float, weighting: str = "derivative",
                fine: int = 2_000_001, seed: int = 0):
    """Quantile grid of p on [0, 1] (trapezoid CDF on a fine grid, then linear
    interpolation of the inverse): x_s = F^-1(q_s) with q_s = (s + 1/2)/N for
    seed 0 (deterministic), or q_s = (s + u_s)/N with u_s the top 53 bits of
    splitmix64(seed + s) scaled to [0, 1) (one point drawn in each of the N
    equal-probability cells; splitmix64 as in ``lanczos.splitmix64``)."""
    g = np.linspace(0.0, 1.0, fine)
    p = _density(g, beta0, mu0, weighting)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (p[1:] + p[:-1]) * np.diff(g))])
    cdf /= cdf[-1]
    if seed == 0:
        q = (np.arange(N) + 0.5) / N
    else:
        from .lanczos import MASK64, splitmix64
        u = np.array([(splitmix64((seed + s) & MASK64) >> 11) * 2.0 ** -53 for s in range(N)])
        q = (np.arange(N) + u) / N
    return np.interp(q, cdf, g)


def forward(theta: np.ndarray, x: np.ndarray, kind: str = "fermi", alpha: float = 1.0,
            mu0: float = 1.0 / 3.0):
    """Model output on samples.  theta has shape (L, 4)."""
    xi = np.asarray(x, dtype=np.float64)
    if kind == "entropy":
        xi = alpha * (xi - mu0) + mu0
    A = np.zeros_like(xi)
    for a, b, c, d in theta:
        A = A + d * xi
        xi = a * xi * xi + b * xi + c
    F = A + xi
    if kind == "entropy":
        return 4.0 * LN2 * F * (1.0 - F)
    return F


def forward_jacobian(theta: np.ndarray, x: np.ndarray, kind: str = "fermi",
                     alpha: float = 1.0, mu0: float = 1.0 / 3.0):
    """Output y (N,) and Jacobian J (N, 4L) of the output w.r.t. the flattened
    table [a_0, b_0, c_0, d_0, a_1, ...], by reverse accumulation:

        g_n = dF/dx_n = 1,   g_i = g_{i+1} (2 a_i x_i + b_i) + d_i,
        dF/da_i = g_{i+1} x_i^2, dF/db_i = g_{i+1} x_i, dF/dc_i = g_{i+1},
        dF/dd_i = x_i,

    (differentiating Eq. mlsp2: x_{i+1} depends on x_i through a x^2 + b x + c,
    A_{i+1} through d x_i, and the output A_n + x_n has unit weight on every
    A_i).  For the entropy model the chain factor 4 ln2 (1 - 2F) multiplies
    every column (Eq. entropy expansion-s)."""
    theta = np.asarray(theta, dtype=np.float64)
    L = theta.shape[0]
    x0 = np.asarray(x, dtype=np.float64)
    xi = alpha * (x0 - mu0) + mu0 if kind == "entropy" else x0.copy()
    xs = [xi]
    A = np.zeros_like(xi)
    for a, b, c, d in theta:
        A = A + d * xs[-1]
        xs.append(a * xs[-1] * xs[-1] + b * xs[-1] + c)
    F = A + xs[-1]
    J = np.empty((x0.size, 4 * L))
    g = np.ones_like(F)            # g_{i+1}, starting at g_n = 1
    for i in range(L - 1, -1, -1):
        a, b, c, d = theta[i]
        xi = xs[i]
        J[:, 4 * i + 0] = g * xi * xi
        J[:, 4 * i + 1] = g * xi
        J[:, 4 * i + 2] = g
        J[:, 4 * i + 3] = xi
        g = g * (2.0 * a * xi + b) + d
    if kind == "entropy":
        fac = 4.0 * LN2 * (1.0 - 2.0 * F)
        return 4.0 * LN2 * F * (1.0 - F), J * fac[:, None]
    return F, J


def target(x, kind: str, beta0: float, mu0: float):
    return entropy_target(x, beta0, mu0) if kind == "entropy" else fermi_target(x, beta0, mu0)


def normal_equations(J: np.ndarray, r: np.ndarray):
    """J^T J and J^T r (the two reductions an LM step needs)."""
    return J.T @ J, J.T @ r


def lm_direction(JTJ: np.ndarray, g: np.ndarray, lam: float):
    """v = -(J^T J + lambda diag(J^T J))^-1 J^T r."""
    M = JTJ + lam * np.diag(np.diag(JTJ))
    return -np.linalg.solve(M, g)


def lm_fit(theta0, x, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, iters=100,
           lam0=1e-3, accel=False, h=0.1, accel_ratio=0.75, callback=None):
    """Plain LM (optionally geodesic-accelerated) on the fixed samples x.
    Returns (theta, history of (cost, lambda, accepted))."""
    theta = np.array(theta0, dtype=np.float64).copy()
    L = theta.shape[0]
    y = target(x, kind, beta0, mu0)
    lam = lam0
    out, J = forward_jacobian(theta, x, kind, alpha, mu0)
    r = out - y
    cost = 0.5 * float(r @ r)
    hist = []
    for it in range(iters):
        JTJ, g = normal_equations(J, r)
        M = JTJ + lam * np.diag(np.diag(JTJ))
        v = -np.linalg.solve(M, g)
        step = v
        if accel:
            rv = forward(theta + h * v.reshape(L, 4), x, kind, alpha, mu0) - y
            rvv = (2.0 / h) * ((rv - r) / h - J @ v)
            a = -np.linalg.solve(M, J.T @ rvv)
            if 2.0 * np.linalg.norm(a) <= accel_ratio * np.linalg.norm(v):
                step = v + 0.5 * a
        cand = theta + step.reshape(L, 4)
        out_c, J_c = forward_jacobian(cand, x, kind, alpha, mu0)
        r_c = out_c - y
        cost_c = 0.5 * float(r_c @ r_c)
        accepted = np.isfinite(cost_c) and cost_c < cost
        if accepted:
            theta, J, r, cost = cand, J_c, r_c, cost_c
            lam = max(lam / 10.0, 1e-12)
        else:
            lam = min(lam * 10.0, 1e12)
        hist.append((cost, lam, accepted))
        if callback is not None:
            callback(it, theta, cost, lam, accepted)
    return theta, hist


def max_error(theta, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, grid=2_000_001):
    """max over an evenly spaced grid on [0, 1] of |model - target|."""
    x = np.linspace(0.0, 1.0, grid)
    return float(np.max(np.abs(forward(np.asarray(theta), x, kind, alpha, mu0)
                               - target(x, kind, beta0, mu0))))


def init_from_sp2(L: int, beta0: float, mu0: float):
    """Initial table (reading of the "scaled and truncated SP2" initial guess,
    Sec. II A 1): the SP2-mu sequence at mu0 (Eq. sp2-mu, Appendix C
    embedding) with an affine contraction x -> mu0 + kappa (x - mu0) folded
    into layer 0 so that the slope at mu0 equals the target's beta0/4
    (kappa <= 1; kappa = 1 when L is below the layer count of Eq. layer count).
    The slope of the composition at mu0 is the product of the layers'
    derivatives 2 a m_i + b along the trajectory m_0 = mu0,
    m_{i+1} = a m_i^2 + b m_i + c (chain rule)."""
    from .sp2 import sp2_table
    th = np.array(sp2_table(mu0, L), dtype=np.float64)
    m, s = mu0, 1.0
    for a, b, c, _ in th:
        s *= 2.0 * a * m + b
        m = a * m * m + b * m + c
    kappa = min(1.0, (beta0 / 4.0) / s)
    m = mu0 * (1.0 - kappa)
    a, b, c, d = th[0]
    th[0] = (a * kappa * kappa, 2 * a * kappa * m + b * kappa, a * m * m + b * m + c, d)
    return th
