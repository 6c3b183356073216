"""The one-term form of the MLSP2 recursion (TEST INFRASTRUCTURE ONLY).

Eq. mlsp2_alt (Sec. II A 1): with t_i = (t_i1, t_i2) for layers i = 0 .. L-1,

    x_{i+1} = (t_i1 + x_i)^2,     A_{i+1} = A_i + t_i2 x_i,

and the output row t_L = (t_L1, t_L2) (Eq. mlsp2_alt-output):

    f(x) ~ A_L + t_L1 + t_L2 x_L.

A table is an array of shape (L + 1, 2); it has 2L + 2 parameters.

Relation to Eq. mlsp2 (Appendix, model embeddings): each layer of this form is
an Eq. mlsp2 layer with (a, b, c, d) = (1, 2 t_i1, t_i1^2, t_i2), and the
output row folds into the last layer: (a, b, c) of layer L-1 scaled by t_L2,
plus t_L1 in c, so that the Eq. mlsp2 output A_L + x_L equals the form's
output.  ``to_mlsp2`` writes this out.  The opposite direction exists
mathematically but needs the per-layer rescaling s_{i+1} = s_i^2 / a_i of the
state, which under- or overflows for general tables (with the printed table s
falls below 1e-300 after ten layers), so tables of this form are trained in
this form (``lm_fit``).

The SP2 sequence (Eq. sp2-mu) is exactly representable: with y = x or
y = 1 - x tracked per layer, x^2 and 2x - x^2 = 1 - (1 - x)^2 are both
(t + y)^2 with t in {0, -1} (``sp2_alt``).
"""
from __future__ import annotations

import numpy as np

from . import train


def alt_scalar(x, alt):
    """Eq. mlsp2_alt and its output row, on an array of layer-0 inputs x."""
    alt = np.asarray(alt, dtype=np.float64)
    L = alt.shape[0] - 1
    y = np.asarray(x, dtype=np.float64).copy()
    A = np.zeros_like(y)
    for i in range(L):
        t1, t2 = alt[i]
        A = A + t2 * y
        y = (t1 + y) * (t1 + y)
    return A + alt[L, 0] + alt[L, 1] * y


def alt_matrix(X0: np.ndarray, alt) -> np.ndarray:
    """The same recursion on a symmetric matrix: X <- (t1 I + X)(t1 I + X)."""
    alt = np.asarray(alt, dtype=np.float64)
    L = alt.shape[0] - 1
    X = np.array(X0, dtype=np.float64)
    I = np.eye(X.shape[0])
    A = np.zeros_like(X)
    for i in range(L):
        t1, t2 = alt[i]
        A = A + t2 * X
        Y = X + t1 * I
        X = Y @ Y
    return A + alt[L, 0] * I + alt[L, 1] * X


def to_mlsp2(alt) -> np.ndarray:
    """Rows (a, b, c, d) of Eq. mlsp2 computing the same function."""
    alt = np.asarray(alt, dtype=np.float64)
    L = alt.shape[0] - 1
    th = np.empty((L, 4))
    for i in range(L):
        t1, t2 = alt[i]
        th[i] = (1.0, 2.0 * t1, t1 * t1, t2)
    w, u = alt[L, 1], alt[L, 0]
    a, b, c, d = th[L - 1]
    th[L - 1] = (w * a, w * b, w * c + u, d)
    return th


def map_jacobian(alt) -> np.ndarray:
    """d theta / d t: (4L, 2L + 2) Jacobian of ``to_mlsp2`` (flattened row-major
    on both sides)."""
    alt = np.asarray(alt, dtype=np.float64)
    L = alt.shape[0] - 1
    P = np.zeros((4 * L, 2 * L + 2))
    for i in range(L):
        t1 = alt[i, 0]
        scale = alt[L, 1] if i == L - 1 else 1.0
        P[4 * i + 1, 2 * i] = 2.0 * scale
        P[4 * i + 2, 2 * i] = 2.0 * t1 * scale
        P[4 * i + 3, 2 * i + 1] = 1.0
    t1 = alt[L - 1, 0]
    P[4 * (L - 1) + 0, 2 * L + 1] = 1.0
    P[4 * (L - 1) + 1, 2 * L + 1] = 2.0 * t1
    P[4 * (L - 1) + 2, 2 * L + 1] = t1 * t1
    P[4 * (L - 1) + 2, 2 * L] = 1.0
    return P


def forward_jacobian(alt, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    """Model output and its Jacobian w.r.t. the 2L + 2 parameters (chain rule
    through ``to_mlsp2``)."""
    F, J = train.forward_jacobian(to_mlsp2(alt), x, kind, alpha, mu0)
    return F, J @ map_jacobian(alt)


def forward(alt, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    if kind == "entropy":
        F = alt_scalar(alpha * (np.asarray(x, dtype=np.float64) - mu0) + mu0, alt)
        return 4.0 * train.LN2 * F * (1.0 - F)
    return alt_scalar(x, alt)


def sp2_alt(mu_p: float, L: int) -> np.ndarray:
    """The SP2 sequence at mu' (Eq. sp2-mu) in this form, no accumulator."""
    from .sp2 import sp2_mu_sequence
    sig, _ = sp2_mu_sequence(mu_p, L)
    alt = np.zeros((L + 1, 2))
    flipped = False             # y = 1 - x when flipped, else y = x
    for i, s in enumerate(sig):
        if s > 0:               # x^2: (0 + y)^2, or (1 - y)^2 = (-1 + y)^2 when flipped
            alt[i, 0] = -1.0 if flipped else 0.0
            flipped = False
        else:                   # 1 - x_{i+1} = (1 - x_i)^2: (-1 + y)^2, or y^2 when flipped
            alt[i, 0] = 0.0 if flipped else -1.0
            flipped = True
    alt[L] = (1.0, -1.0) if flipped else (0.0, 1.0)
    return alt


def lm_fit(alt0, x, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, iters=100, lam0=1e-3,
           accel=False, h=0.1, accel_ratio=0.75):
    """Levenberg-Marquardt on the 2L + 2 parameters, the same update and
    acceptance rules as ``train.lm_fit``."""
    p = np.array(alt0, dtype=np.float64).copy()
    shape = p.shape
    y = train.target(x, kind, beta0, mu0)
    out, J = forward_jacobian(p, x, kind, alpha, mu0)
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
            rv = forward(p + h * v.reshape(shape), x, kind, alpha, mu0) - y
            rvv = (2.0 / h) * ((rv - r) / h - J @ v)
            acc = -np.linalg.solve(M, J.T @ rvv)
            if 2.0 * np.linalg.norm(acc) <= accel_ratio * np.linalg.norm(v):
                step = v + 0.5 * acc
        cand = p + step.reshape(shape)
        out_c, J_c = forward_jacobian(cand, x, kind, alpha, mu0)
        r_c = out_c - y
        cost_c = 0.5 * float(r_c @ r_c)
        ok = np.isfinite(cost_c) and cost_c < cost
        if ok:
            p, J, r, cost = cand, J_c, r_c, cost_c
            lam = max(lam / 10.0, 1e-12)
        else:
            lam = min(lam * 10.0, 1e12)
        hist.append((cost, lam, ok))
    return p, hist


def max_error(alt, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, grid=2_000_001):
    x = np.linspace(0.0, 1.0, grid)
    return float(np.max(np.abs(forward(alt, x, kind, alpha, mu0) - train.target(x, kind, beta0, mu0))))


def method_exact(H: np.ndarray, mu: float, kT: float, alt, beta0: float, mu0: float, alpha: float,
                 alt_entropy=None):
    """D_rec and S_rec for one table of this form: the rescaling of
    ``rescale.rescale`` (Gershgorin bounds, flip), the scalar recursion of Eq.
    mlsp2_alt on the mapped eigenvalues, D = V diag(P) V^T (1 - P when flipped)
    and S = sum of 4 ln2 F (1 - F) with the entropy table (or the Fermi table
    when none is given) started at alpha (x0 - mu0) + mu0."""
    from . import rescale
    alt = np.asarray(alt, dtype=np.float64)
    L = alt.shape[0] - 1
    meta = rescale.Table(tuple((0.0, 0.0, 0.0, 0.0) for _ in range(L)), beta0, mu0, alpha)
    H0, rec = rescale.rescale(H, mu, kT, [meta])
    if H0 is None:
        return dict(D=None, S=None, rec=rec)
    eps, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    x0 = rescale.x0_of_eigenvalue(eps, mu, kT, rec, meta)
    p = alt_scalar(x0, alt)
    if rec.flip:
        p = 1.0 - p
    D = (V * p[None, :]) @ V.T
    ent = alt if alt_entropy is None else np.asarray(alt_entropy, dtype=np.float64)
    s = forward(ent, x0, "entropy", alpha, mu0)
    return dict(D=D, S=float(np.sum(s)), trD=float(np.sum(p)), rec=rec, x0=x0)
