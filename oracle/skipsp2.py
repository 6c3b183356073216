"""Skip-SP2 with one stored layer and one accumulator (TEST INFRASTRUCTURE ONLY).

Sec. II A 3 (recombinant layers and accumulators), with k = 1 stored layer
and K = 1 accumulator, and the initial accumulator constant A_0 and output
weight of the Appendix's embeddings.  A table has L layer rows
(delta_i, alpha_i, beta_i, gamma_i) and one output row (A_0, gamma_L):

    u_i     = delta_i + alpha_i x_i + beta_i A_i
    A_{i+1} = A_i + gamma_i x_i
    x_{i+1} = u_i^2                                   (i = 0 .. L-1)

    f(x) ~ A_L + gamma_L x_L,        A_0 = the output row's first entry,

on the layer-0 input x_0 = x (no inner flip, like the Eq. mlsp2 tables).
In the paper's notation delta_i = alpha_{i,k}, alpha_i = alpha_{i,0},
beta_i = beta_{i,1}.  The accumulator feeding back into the squared
combination (beta_i != 0) is what this family adds over Eq. mlsp2: every
earlier layer reaches layer i + 1 through A_i.  Array shape (L + 1, 4); the
output row stores (A_0, gamma_L, 0, 0); 4L + 2 parameters.

``from_mlsp2`` is the Appendix's embedding of Eq. mlsp2 (beta = 0): with
e_i = c_i - b_i^2 / (4 a_i), the squared combinations are
x~_{i+1} = (x_i + b_i / (2 a_i))^2 and x_{i+1} = a_i x~_{i+1} + e_i, so
alpha_0 = 1, delta_0 = b_0 / (2 a_0), alpha_i = a_{i-1},
delta_i = e_{i-1} + b_i / (2 a_i); gamma_0 = d_0, gamma_i = d_i a_{i-1},
gamma_L = a_{L-1} and A_0 = sum_{i=1}^{L-1} d_i e_{i-1} + e_{L-1}.
"""
from __future__ import annotations

import numpy as np

from . import train


def skip_scalar(x, tab):
    """The recursion and its output on an array of layer-0 inputs."""
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    xi = np.asarray(x, dtype=np.float64).copy()
    A = np.full_like(xi, tab[L, 0])
    for i in range(L):
        dl, al, be, ga = tab[i]
        u = dl + al * xi + be * A
        A = A + ga * xi
        xi = u * u
    return A + tab[L, 1] * xi


def skip_matrix(X0: np.ndarray, tab) -> np.ndarray:
    """The same recursion on a symmetric matrix: U = delta I + alpha X + beta A,
    X <- U U."""
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    X = np.array(X0, dtype=np.float64)
    I = np.eye(X.shape[0])
    A = tab[L, 0] * I
    for i in range(L):
        dl, al, be, ga = tab[i]
        U = dl * I + al * X + be * A
        A = A + ga * X
        X = U @ U
    return A + tab[L, 1] * X


def from_mlsp2(theta) -> np.ndarray:
    """The Appendix's embedding of an Eq. mlsp2 table (rows a, b, c, d)."""
    th = np.asarray(theta, dtype=np.float64)
    L = th.shape[0]
    tab = np.zeros((L + 1, 4))
    e = th[:, 2] - th[:, 1] ** 2 / (4.0 * th[:, 0])
    for i in range(L):
        a, b, _, d = th[i]
        if i == 0:
            tab[i] = (b / (2.0 * a), 1.0, 0.0, d)
        else:
            tab[i] = (e[i - 1] + b / (2.0 * a), th[i - 1, 0], 0.0, d * th[i - 1, 0])
    A0 = e[L - 1] + sum(th[i, 3] * e[i - 1] for i in range(1, L))
    tab[L] = (A0, th[L - 1, 0], 0.0, 0.0)
    return tab


def forward_jacobian(tab, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    """Output and Jacobian (N, 4L + 2) w.r.t. (delta_0, alpha_0, beta_0,
    gamma_0, ..., A_0, gamma_L) by reverse accumulation: with gx_i = dF/dx_i
    and gA_i = dF/dA_i, gx_L = gamma_L, gA_L = 1, and for i = L-1 .. 0
    (w = 2 u_i gx_{i+1}):
        dF/d delta_i = w, dF/d alpha_i = w x_i, dF/d beta_i = w A_i,
        dF/d gamma_i = gA_{i+1} x_i,
        gx_i = w alpha_i + gA_{i+1} gamma_i,   gA_i = w beta_i + gA_{i+1};
    dF/dA_0 = gA_0 and dF/d gamma_L = x_L.  The entropy model multiplies every
    column by 4 ln2 (1 - 2F)."""
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    x0 = np.asarray(x, dtype=np.float64)
    xi = alpha * (x0 - mu0) + mu0 if kind == "entropy" else x0.copy()
    xs, As, us = [xi], [np.full_like(xi, tab[L, 0])], []
    for i in range(L):
        dl, al, be, ga = tab[i]
        u = dl + al * xs[-1] + be * As[-1]
        us.append(u)
        As.append(As[-1] + ga * xs[-1])
        xs.append(u * u)
    F = As[-1] + tab[L, 1] * xs[-1]
    J = np.empty((x0.size, 4 * L + 2))
    gx = np.full_like(F, tab[L, 1])
    gA = np.ones_like(F)
    J[:, 4 * L + 1] = xs[-1]
    for i in range(L - 1, -1, -1):
        dl, al, be, ga = tab[i]
        w = 2.0 * us[i] * gx
        J[:, 4 * i + 0] = w
        J[:, 4 * i + 1] = w * xs[i]
        J[:, 4 * i + 2] = w * As[i]
        J[:, 4 * i + 3] = gA * xs[i]
        gx, gA = w * al + gA * ga, w * be + gA
    J[:, 4 * L] = gA
    if kind == "entropy":
        fac = 4.0 * train.LN2 * (1.0 - 2.0 * F)
        return 4.0 * train.LN2 * F * (1.0 - F), J * fac[:, None]
    return F, J


def forward(tab, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    if kind == "entropy":
        F = skip_scalar(alpha * (np.asarray(x, dtype=np.float64) - mu0) + mu0, tab)
        return 4.0 * train.LN2 * F * (1.0 - F)
    return skip_scalar(x, tab)


def _flat(tab):
    tab = np.asarray(tab, dtype=np.float64)
    return np.concatenate([tab[:-1].ravel(), tab[-1, :2]])


def _unflat(p, L):
    tab = np.zeros((L + 1, 4))
    tab[:L] = p[:4 * L].reshape(L, 4)
    tab[L, :2] = p[4 * L:]
    return tab


def lm_fit(tab0, x, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, iters=100, lam0=1e-3, accel=False,
           h=0.1, accel_ratio=0.75):
    """Levenberg-Marquardt on the 4L + 2 parameters, the update and acceptance
    rules of ``train.lm_fit``."""
    tab0 = np.asarray(tab0, dtype=np.float64)
    L = tab0.shape[0] - 1
    p = _flat(tab0)
    y = train.target(x, kind, beta0, mu0)
    out, J = forward_jacobian(_unflat(p, L), x, kind, alpha, mu0)
    r = out - y
    cost = 0.5 * float(r @ r)
    lam = lam0
    hist = []
    for _ in range(iters):
        JTJ, g = train.normal_equations(J, r)
        M = JTJ + lam * np.diag(np.diag(JTJ))
        v = -np.linalg.solve(M, g)
        step = v
        if accel:
            rv = forward(_unflat(p + h * v, L), x, kind, alpha, mu0) - y
            rvv = (2.0 / h) * ((rv - r) / h - J @ v)
            acc = -np.linalg.solve(M, J.T @ rvv)
            if 2.0 * np.linalg.norm(acc) <= accel_ratio * np.linalg.norm(v):
                step = v + 0.5 * acc
        cand = p + step
        out_c, J_c = forward_jacobian(_unflat(cand, L), x, kind, alpha, mu0)
        r_c = out_c - y
        cost_c = 0.5 * float(r_c @ r_c)
        ok = np.isfinite(cost_c) and cost_c < cost
        if ok:
            p, J, r, cost = cand, J_c, r_c, cost_c
            lam = max(lam / 10.0, 1e-12)
        else:
            lam = min(lam * 10.0, 1e12)
        hist.append((cost, lam, ok))
    return _unflat(p, L), hist


def max_error(tab, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, grid=2_000_001):
    x = np.linspace(0.0, 1.0, grid)
    return float(np.max(np.abs(forward(tab, x, kind, alpha, mu0) - train.target(x, kind, beta0, mu0))))


def method_exact(H: np.ndarray, mu: float, kT: float, tab, beta0: float, mu0: float, alpha: float, tab_entropy=None):
    """D_rec and S_rec for one table of this family (the rescaling of
    ``rescale.rescale``; the scalar recursion on the mapped eigenvalues)."""
    from . import rescale
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    meta = rescale.Table(tuple((0.0, 0.0, 0.0, 0.0) for _ in range(L)), beta0, mu0, alpha)
    H0, rec = rescale.rescale(H, mu, kT, [meta])
    if H0 is None:
        return dict(D=None, S=None, rec=rec)
    eps, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    x0 = rescale.x0_of_eigenvalue(eps, mu, kT, rec, meta)
    p = skip_scalar(x0, tab)
    if rec.flip:
        p = 1.0 - p
    D = (V * p[None, :]) @ V.T
    ent = tab if tab_entropy is None else np.asarray(tab_entropy, dtype=np.float64)
    s = forward(ent, x0, "entropy", alpha, mu0)
    return dict(D=D, S=float(np.sum(s)), trD=float(np.sum(p)), rec=rec, x0=x0)
