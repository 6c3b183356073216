"""Max-SP2, and Skip-SP2 with k stored layers and K accumulators
(TEST INFRASTRUCTURE ONLY).

Max-SP2 (Sec. II A 2, Eq. maxsp2): every layer squares an affine combination
of all the layers before it,

    x_0 = x,   u_i = delta_i + sum_{j=0}^{i} theta_{i,j} x_j,   x_{i+1} = u_i^2
    (i = 0 .. L-1),        f(x) ~ c + sum_{j=0}^{L} gamma_j x_j,

on the layer-0 input x_0 = x (no inner flip, like every table here).
Reading: Eq. maxsp2 accumulates A_{i+1} = A_i + gamma_i x_i from A_0 = 0 and
outputs A_L + gamma_L x_L = sum_j gamma_j x_j; Alg. maxsp2 outputs
gamma_0 + sum_{i >= 1} gamma_i x_i, a constant in place of the x_0 term.  The
form above holds both (c = 0, or gamma_0 = 0 with c the constant).

Flat layout of a table (the library's too): for i = 0 .. L-1 the block
(delta_i, gamma_i, theta_{i,0}, ..., theta_{i,i}), then (c, gamma_L):
L (L + 5) / 2 + 2 numbers.

Skip-SP2 (Sec. II A 3) with k stored layers and K accumulators:

    u_i       = alpha_{i,k} + sum_{j=0}^{min(k-1, i)} alpha_{i,j} x_{i-j}
                + sum_{l=1}^{K} beta_{i,l} A_{i,l}
    A_{i+1,l} = A_{i,l} + gamma_{i,l} x_i,    x_{i+1} = u_i^2,
    f(x) ~ gamma_L x_L + sum_l A_{L,l},      A_{0,l} given.

A table is a dict of arrays: alpha (L, k + 1) with the constant alpha_{i,k}
last, beta (L, K), gamma (L, K), A0 (K,), and the output weight gL.
Reading: the paper writes the output as x_L + sum_l A_{L,l} (gL = 1) and counts
(1 + k + 2K) L + 2 parameters, two beyond the layers' own; the Appendix's
embedding of Eq. mlsp2 needs an output weight a_{L-1} on the last layer (its
accumulator sum runs to i = L), so the two are read as A_0 and gL, the
layout of the one-accumulator tables (output row (A_0, gamma_L)).

Embedding in Max-SP2 (the Appendix's Skip-SP2 in Max-SP2, written out from
the definitions): A_{i,l} = A_{0,l} + sum_{j<i} gamma_{j,l} x_j, so

    delta_i       = alpha_{i,k} + sum_l beta_{i,l} A_{0,l},
    theta_{i,j}   = sum_l beta_{i,l} gamma_{j,l} [j < i] + alpha_{i,i-j} [i - j < k],
    c = sum_l A_{0,l},   gamma_j = sum_l gamma_{j,l} (j < L),   gamma_L = gL.

(The Appendix prints the accumulator term for every j <= i; gamma_{i,l} x_i
only enters A_{i+1,l}, so it belongs to the layers after i.)
"""
from __future__ import annotations

import numpy as np

from . import skipsp2, train


def nparams(L: int) -> int:
    return L * (L + 5) // 2 + 2


def unflat(p, L):
    """(delta (L,), gamma (L + 1,), theta (list of L arrays, theta[i] of i + 1), c)."""
    p = np.asarray(p, dtype=np.float64)
    assert p.size == nparams(L)
    delta, gamma, theta = np.zeros(L), np.zeros(L + 1), []
    o = 0
    for i in range(L):
        delta[i], gamma[i] = p[o], p[o + 1]
        theta.append(p[o + 2:o + 3 + i].copy())
        o += i + 3
    c, gamma[L] = p[o], p[o + 1]
    return delta, gamma, theta, c


def flat(delta, gamma, theta, c):
    out = []
    for i in range(len(delta)):
        out += [delta[i], gamma[i]] + list(theta[i])
    out += [c, gamma[len(delta)]]
    return np.array(out, dtype=np.float64)


def max_scalar(x, p, L):
    """The recursion of Eq. maxsp2 and its output on an array of layer-0 inputs."""
    delta, gamma, theta, c = unflat(p, L)
    xs = [np.asarray(x, dtype=np.float64).copy()]
    for i in range(L):
        u = delta[i] + sum(theta[i][j] * xs[j] for j in range(i + 1))
        xs.append(u * u)
    return c + sum(gamma[j] * xs[j] for j in range(L + 1))


def max_matrix(X0: np.ndarray, p, L) -> np.ndarray:
    """The same recursion on a symmetric matrix: U_i = delta_i I + sum_j theta_{i,j} X_j,
    X_{i+1} = U_i U_i; output c I + sum_j gamma_j X_j."""
    delta, gamma, theta, c = unflat(p, L)
    X0 = np.array(X0, dtype=np.float64)
    I = np.eye(X0.shape[0])
    Xs = [X0]
    for i in range(L):
        U = delta[i] * I + sum(theta[i][j] * Xs[j] for j in range(i + 1))
        Xs.append(U @ U)
    return c * I + sum(gamma[j] * Xs[j] for j in range(L + 1))


def skip_scalar(x, t):
    """Skip-SP2 with k stored layers and K accumulators (table dict t)."""
    alpha, beta, gamma, A0 = (np.asarray(t[k], dtype=np.float64) for k in ("alpha", "beta", "gamma", "A0"))
    L, k = alpha.shape[0], alpha.shape[1] - 1
    K = beta.shape[1]
    xs = [np.asarray(x, dtype=np.float64).copy()]
    A = [np.full_like(xs[0], A0[l]) for l in range(K)]
    for i in range(L):
        u = alpha[i, k] + sum(alpha[i, j] * xs[i - j] for j in range(min(k - 1, i) + 1))
        u = u + sum(beta[i, l] * A[l] for l in range(K))
        A = [A[l] + gamma[i, l] * xs[i] for l in range(K)]
        xs.append(u * u)
    return float(t.get("gL", 1.0)) * xs[L] + sum(A)


def skip_matrix(X0: np.ndarray, t) -> np.ndarray:
    alpha, beta, gamma, A0 = (np.asarray(t[k], dtype=np.float64) for k in ("alpha", "beta", "gamma", "A0"))
    L, k = alpha.shape[0], alpha.shape[1] - 1
    K = beta.shape[1]
    X0 = np.array(X0, dtype=np.float64)
    I = np.eye(X0.shape[0])
    Xs = [X0]
    A = [A0[l] * I for l in range(K)]
    for i in range(L):
        U = alpha[i, k] * I + sum(alpha[i, j] * Xs[i - j] for j in range(min(k - 1, i) + 1))
        U = U + sum(beta[i, l] * A[l] for l in range(K))
        A = [A[l] + gamma[i, l] * Xs[i] for l in range(K)]
        Xs.append(U @ U)
    return float(t.get("gL", 1.0)) * Xs[L] + sum(A)


def skip_to_max(t):
    """Flat Max-SP2 table computing the same function as the Skip-SP2 table t."""
    alpha, beta, gamma, A0 = (np.asarray(t[k], dtype=np.float64) for k in ("alpha", "beta", "gamma", "A0"))
    L, k = alpha.shape[0], alpha.shape[1] - 1
    K = beta.shape[1]
    delta = np.array([alpha[i, k] + sum(beta[i, l] * A0[l] for l in range(K)) for i in range(L)])
    theta = []
    for i in range(L):
        th = np.zeros(i + 1)
        for j in range(i + 1):
            if j < i:
                th[j] += sum(beta[i, l] * gamma[j, l] for l in range(K))
            if i - j < k:
                th[j] += alpha[i, i - j]
        theta.append(th)
    g = np.zeros(L + 1)
    g[:L] = [sum(gamma[j, l] for l in range(K)) for j in range(L)]
    g[L] = float(t.get("gL", 1.0))
    return flat(delta, g, theta, float(np.sum(A0)))


def skip1_to_max(tab):
    """Flat Max-SP2 table of a Skip-SP2 table with one stored layer and one
    accumulator in the (L + 1, 4) layout of ``skipsp2`` (rows (delta, alpha,
    beta, gamma), output row (A_0, gamma_L)): u_i = delta_i + alpha_i x_i +
    beta_i (A_0 + sum_{j<i} gamma_j x_j), output A_0 + sum_{j<L} gamma_j x_j +
    gamma_L x_L."""
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    A0, gL = tab[L, 0], tab[L, 1]
    delta = tab[:L, 0] + tab[:L, 2] * A0
    theta = []
    for i in range(L):
        th = tab[i, 2] * tab[:i, 3]
        theta.append(np.concatenate([th, [tab[i, 1]]]))
    g = np.concatenate([tab[:L, 3], [gL]])
    return flat(delta, g, theta, A0)


def mlsp2_to_max(theta):
    """Flat Max-SP2 table of Eq. mlsp2 rows, through the Appendix's embedding
    of Eq. mlsp2 in Skip-SP2 (``skipsp2.from_mlsp2``)."""
    return skip1_to_max(skipsp2.from_mlsp2(theta))


def forward_jacobian(p, L, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    """Output and Jacobian (N, nparams(L)) w.r.t. the flat table by reverse
    accumulation: with g_j = dF/dx_j, g_j starts at gamma_j, and for
    i = L-1 .. 0 (w = 2 u_i g_{i+1}, g_{i+1} final once the layers after i
    are done):
        dF/d delta_i = w,   dF/d theta_{i,j} = w x_j,   g_j += w theta_{i,j} (j <= i);
    dF/d gamma_j = x_j, dF/dc = 1.  The entropy model multiplies every column
    by 4 ln2 (1 - 2F)."""
    delta, gamma, theta, c = unflat(p, L)
    x0 = np.asarray(x, dtype=np.float64)
    xi = alpha * (x0 - mu0) + mu0 if kind == "entropy" else x0.copy()
    xs, us = [xi], []
    for i in range(L):
        u = delta[i] + sum(theta[i][j] * xs[j] for j in range(i + 1))
        us.append(u)
        xs.append(u * u)
    F = c + sum(gamma[j] * xs[j] for j in range(L + 1))
    J = np.zeros((x0.size, nparams(L)))
    g = [np.full_like(F, gamma[j]) for j in range(L + 1)]
    offs, o = [], 0
    for i in range(L):
        offs.append(o)
        o += i + 3
    J[:, o] = 1.0
    J[:, o + 1] = xs[L]
    for i in range(L - 1, -1, -1):
        w = 2.0 * us[i] * g[i + 1]
        J[:, offs[i]] = w
        J[:, offs[i] + 1] = xs[i]
        for j in range(i + 1):
            J[:, offs[i] + 2 + j] = w * xs[j]
            g[j] = g[j] + w * theta[i][j]
    if kind == "entropy":
        fac = 4.0 * train.LN2 * (1.0 - 2.0 * F)
        return 4.0 * train.LN2 * F * (1.0 - F), J * fac[:, None]
    return F, J


def forward(p, L, x, kind="fermi", alpha=1.0, mu0=1.0 / 3.0):
    if kind == "entropy":
        F = max_scalar(alpha * (np.asarray(x, dtype=np.float64) - mu0) + mu0, p, L)
        return 4.0 * train.LN2 * F * (1.0 - F)
    return max_scalar(x, p, L)


def lm_fit(p0, L, x, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, iters=100, lam0=1e-3, accel=False,
           h=0.1, accel_ratio=0.75):
    """Levenberg-Marquardt on the flat table, the update and acceptance rules
    of ``train.lm_fit``."""
    p = np.array(p0, dtype=np.float64)
    y = train.target(x, kind, beta0, mu0)
    out, J = forward_jacobian(p, L, x, kind, alpha, mu0)
    r = out - y
    cost = 0.5 * float(r @ r)
    lam = lam0
    hist = []
    for _ in range(iters):
        JTJ, gr = train.normal_equations(J, r)
        M = JTJ + lam * np.diag(np.diag(JTJ))
        try:
            v = -np.linalg.solve(M, gr)
        except np.linalg.LinAlgError:
            lam = min(lam * 10.0, 1e12)
            hist.append((cost, lam, False))
            continue
        step = v
        if accel:
            rv = forward(p + h * v, L, x, kind, alpha, mu0) - y
            rvv = (2.0 / h) * ((rv - r) / h - J @ v)
            acc = -np.linalg.solve(M, J.T @ rvv)
            if 2.0 * np.linalg.norm(acc) <= accel_ratio * np.linalg.norm(v):
                step = v + 0.5 * acc
        cand = p + step
        out_c, J_c = forward_jacobian(cand, L, x, kind, alpha, mu0)
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


def skip_pack(t):
    """Trainable parameters of a Skip-SP2 table dict: alpha, beta, gamma
    (row-major), A_{0,1} and gL, (1 + k + 2K) L + 2 numbers, the paper's
    count.  The other initial accumulators stay zero (their values only add
    beta-weighted constants that alpha_{i,k} already holds, and the output's
    constant is A_{0,1})."""
    A0 = np.asarray(t["A0"], dtype=np.float64).ravel()
    assert np.all(A0[1:] == 0.0)
    return np.concatenate([np.asarray(t[k], dtype=np.float64).ravel() for k in ("alpha", "beta", "gamma")]
                          + [A0[:1], np.array([float(t.get("gL", 1.0))])])


def skip_unpack(q, L, k, K):
    q = np.asarray(q, dtype=np.float64)
    na, nbg = L * (k + 1), L * K
    A0 = np.zeros(K)
    A0[0] = q[na + 2 * nbg]
    return dict(alpha=q[:na].reshape(L, k + 1), beta=q[na:na + nbg].reshape(L, K),
                gamma=q[na + nbg:na + 2 * nbg].reshape(L, K), A0=A0, gL=float(q[na + 2 * nbg + 1]))


def skip_embedding_jacobian(q, L, k, K):
    """d skip_to_max / d q (nparams(L) x len(q)).  Every Max-SP2 entry is
    affine in each single Skip-SP2 parameter (the products beta gamma are
    bilinear), so a central difference with a unit step is the derivative up
    to rounding."""
    q = np.asarray(q, dtype=np.float64)
    E = np.zeros((nparams(L), q.size))
    for m in range(q.size):
        e = np.zeros_like(q)
        e[m] = 1.0
        E[:, m] = 0.5 * (skip_to_max(skip_unpack(q + e, L, k, K)) - skip_to_max(skip_unpack(q - e, L, k, K)))
    return E


def skip_lm_fit(t0, kind="fermi", x=None, beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, iters=100, lam0=1e-3,
                accel=False, h=0.1, accel_ratio=0.75):
    """Levenberg-Marquardt on a Skip-SP2 table with k stored layers and K
    accumulators (Sec. II C 2 applied to the family of Sec. II A 3).  The
    output is the Max-SP2 output of the table's embedding, so its Jacobian is
    the Max-SP2 Jacobian times the embedding's (chain rule); the update and
    acceptance rules are those of ``lm_fit``, with one reading: a zero
    diagonal entry of J^T J (a parameter the output does not depend on at the
    current point, e.g. the feedback of an accumulator that is still zero) is
    raised to the smallest positive one before damping, so that the damped
    matrix stays regular; such a parameter takes no step until it matters."""
    L, k, K = np.asarray(t0["alpha"]).shape[0], np.asarray(t0["alpha"]).shape[1] - 1, np.asarray(t0["beta"]).shape[1]
    q = skip_pack(t0)
    y = train.target(x, kind, beta0, mu0)

    def fj(qq):
        out, Jm = forward_jacobian(skip_to_max(skip_unpack(qq, L, k, K)), L, x, kind, alpha, mu0)
        return out, Jm @ skip_embedding_jacobian(qq, L, k, K)

    out, J = fj(q)
    r = out - y
    cost = 0.5 * float(r @ r)
    lam = lam0
    hist = []
    for _ in range(iters):
        JTJ, gr = train.normal_equations(J, r)
        dg = np.diag(JTJ).copy()
        pos = dg[dg > 0.0]
        dg[dg <= 0.0] = pos.min() if pos.size else 1.0
        M = JTJ + lam * np.diag(dg)
        try:
            v = -np.linalg.solve(M, gr)
        except np.linalg.LinAlgError:
            lam = min(lam * 10.0, 1e12)
            hist.append((cost, lam, False))
            continue
        step = v
        if accel:
            rv = forward(skip_to_max(skip_unpack(q + h * v, L, k, K)), L, x, kind, alpha, mu0) - y
            rvv = (2.0 / h) * ((rv - r) / h - J @ v)
            acc = -np.linalg.solve(M, J.T @ rvv)
            if 2.0 * np.linalg.norm(acc) <= accel_ratio * np.linalg.norm(v):
                step = v + 0.5 * acc
        cand = q + step
        out_c, J_c = fj(cand)
        r_c = out_c - y
        cost_c = 0.5 * float(r_c @ r_c)
        ok = np.isfinite(cost_c) and cost_c < cost
        if ok:
            q, J, r, cost = cand, J_c, r_c, cost_c
            lam = max(lam / 10.0, 1e-12)
        else:
            lam = min(lam * 10.0, 1e12)
        hist.append((cost, lam, ok))
    return skip_unpack(q, L, k, K), hist


def skip_from_skip1(tab, k, K, beta_extra=0.0):
    """A Skip-SP2 table with one stored layer and one accumulator ((L + 1, 4)
    rows of ``skipsp2``) as a table with k >= 1 stored layers and K >= 1
    accumulators computing the same function: the extra stored-layer weights
    and the extra accumulators' inputs gamma start at zero (the output sums
    every accumulator, so they must); the extra accumulators' feedback beta
    start at beta_extra (no effect while those accumulators stay zero;
    nonzero gives their gamma a derivative through the layers as well)."""
    tab = np.asarray(tab, dtype=np.float64)
    L = tab.shape[0] - 1
    alpha, beta, gamma, A0 = np.zeros((L, k + 1)), np.zeros((L, K)), np.zeros((L, K)), np.zeros(K)
    alpha[:, 0], alpha[:, k] = tab[:L, 1], tab[:L, 0]
    beta[:, 0], gamma[:, 0] = tab[:L, 2], tab[:L, 3]
    beta[:, 1:] = beta_extra
    A0[0] = tab[L, 0]
    return dict(alpha=alpha, beta=beta, gamma=gamma, A0=A0, gL=float(tab[L, 1]))


def max_error(p, L, kind="fermi", beta0=1500.0, mu0=1.0 / 3.0, alpha=1.0, grid=2_000_001):
    x = np.linspace(0.0, 1.0, grid)
    return float(np.max(np.abs(forward(p, L, x, kind, alpha, mu0) - train.target(x, kind, beta0, mu0))))


def method_exact(H: np.ndarray, mu: float, kT: float, p, L, beta0: float, mu0: float, alpha: float,
                 p_entropy=None, L_entropy=None):
    """D_rec and S_rec for one Max-SP2 table (the rescaling of
    ``rescale.rescale``; the scalar recursion on the mapped eigenvalues)."""
    from . import rescale
    meta = rescale.Table(tuple((0.0, 0.0, 0.0, 0.0) for _ in range(L)), beta0, mu0, alpha)
    H0, rec = rescale.rescale(H, mu, kT, [meta])
    if H0 is None:
        return dict(D=None, S=None, rec=rec)
    eps, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    x0 = rescale.x0_of_eigenvalue(eps, mu, kT, rec, meta)
    f = max_scalar(x0, p, L)
    if rec.flip:
        f = 1.0 - f
    D = (V * f[None, :]) @ V.T
    pe, Le = (p, L) if p_entropy is None else (p_entropy, L_entropy)
    s = forward(pe, Le, x0, "entropy", alpha, mu0)
    return dict(D=D, S=float(np.sum(s)), trD=float(np.sum(f)), rec=rec, x0=x0)
