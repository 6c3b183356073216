"""Spectral bounds from a few Lanczos steps, intersected with the Gershgorin
bounds (TEST INFRASTRUCTURE ONLY).

The paper bounds the spectrum with Gershgorin circles (Appendix A) and notes
Lanczos estimates of the eigenvalues near the Fermi level (Sec. II B).  A
tighter interval [e_min, e_max] shrinks W, hence beta' = W beta (Eq. beta'), the
beta0 a model needs, its layer count (Eq. layer count) and the amplification of
rounding.  Steps, in order:

1. start vector: q_i = 2 u_i - 1, u_i the top 53 bits of splitmix64(i) scaled to
   [0, 1) (splitmix64: Steele, Lea and Flood, OOPSLA 2014; i = 0 .. n-1), then
   v_1 = q / ||q||;
2. k = min(n, K_STEPS) steps of the three-term Lanczos recurrence in FP64
   without re-orthogonalisation:
       w = H v_j - beta_{j-1} v_{j-1},  alpha_j = w . v_j,  w <- w - alpha_j v_j,
       beta_j = ||w||,  v_{j+1} = w / beta_j,
   stopping early when beta_j <= 1e-12 * (|alpha_1| + beta_1 + 1) (an invariant
   subspace: the Ritz values are eigenvalues);
3. the extreme eigenvalues theta_min, theta_max of the tridiagonal T_k and the
   residual bounds r = beta_k |s_k| of their Ritz pairs (s the normalised
   eigenvector of T_k; r = 0 after an early stop);
4. lo = theta_min - r_min - delta, hi = theta_max + r_max + delta with
   delta = MARGIN * (theta_max - theta_min);
5. e_min = max(gershgorin_min, lo), e_max = min(gershgorin_max, hi), each kept
   inside the Gershgorin interval so that e_min <= e_max.

Readings (the paper fixes none of this): K_STEPS = 24, MARGIN = 1e-2, no
re-orthogonalisation, the residual bound of step 3 as the safety term.  The
interval is not a rigorous enclosure: the pins check that it contains the
spectrum of every workload family used here.  This is the FP64 definition of
the bounds and nothing in it depends on how an implementation rounds; an
implementation that forms the products H v in lower precision moves the
interval by its own rounding, which its tests bound separately.
"""
from __future__ import annotations

import numpy as np

from . import rescale

K_STEPS = 24
MARGIN = 1e-2
MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of splitmix64 for state x (the generator's published
    definition: add the golden-gamma constant, then two xor-shift-multiply
    rounds and a final xor-shift)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def start_vector(n: int) -> np.ndarray:
    q = np.array([2.0 * ((splitmix64(i) >> 11) * 2.0 ** -53) - 1.0 for i in range(n)])
    return q / np.linalg.norm(q)


def lanczos_tridiagonal(H: np.ndarray, k: int):
    """(alpha[0..m-1], beta[0..m-1]) of m <= k Lanczos steps from start_vector;
    beta[m-1] is the coupling to the next (unformed) vector."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    v_prev = np.zeros(n)
    v = start_vector(n)
    alphas, betas = [], []
    beta_prev = 0.0
    for _ in range(min(k, n)):
        w = H @ v - beta_prev * v_prev
        a = float(w @ v)
        w = w - a * v
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        if b <= 1e-12 * (abs(alphas[0]) + betas[0] + 1.0):
            break
        v_prev, v, beta_prev = v, w / b, b
    return np.array(alphas), np.array(betas)


def ritz_extremes(alphas: np.ndarray, betas: np.ndarray):
    """(theta_min, r_min, theta_max, r_max) of the tridiagonal T (diagonal
    alphas, off-diagonal betas[:-1]); r = beta_last * |last eigenvector entry|."""
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    theta, S = np.linalg.eigh(T)
    b_last = betas[-1]
    return (float(theta[0]), float(b_last * abs(S[m - 1, 0])),
            float(theta[-1]), float(b_last * abs(S[m - 1, -1])))


def bounds(H: np.ndarray, k: int = K_STEPS, margin: float = MARGIN):
    """(e_min, e_max): the Lanczos interval of steps 1-4 intersected with the
    Gershgorin interval (step 5)."""
    g_lo, g_hi = rescale.gershgorin(H)
    alphas, betas = lanczos_tridiagonal(H, k)
    t_lo, r_lo, t_hi, r_hi = ritz_extremes(alphas, betas)
    delta = margin * (t_hi - t_lo)
    lo, hi = t_lo - r_lo - delta, t_hi + r_hi + delta
    return max(g_lo, min(lo, g_hi)), min(g_hi, max(hi, g_lo))
