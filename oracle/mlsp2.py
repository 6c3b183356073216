"""MLSP2 recursions, scalar and matrix (TEST INFRASTRUCTURE ONLY).

A coefficient table ``theta`` is a sequence of rows (a, b, c, d) =
(theta_i1, theta_i2, theta_i3, theta_i4).  Layer i (Eq. mlsp2, Sec. II A 1):

    A_{i+1} = A_i + d_i x_i
    x_{i+1} = a_i x_i^2 + b_i x_i + c_i

and the output is A_n + x_n (Eq. mlsp2-output).  Readings:

* The accumulator takes the layer input x_i, before that layer's quadratic
  update (Eq. mlsp2 and Alg. 1 order; Alg. 2's loop does the same).
* No inner flip x0 = 1 - x: the input x is the layer-0 value itself.  The
  Appendix A program applies no inner flip, and the printed weights only
  approximate the Fermi function under this convention (pinned by the tests).
* The constant c_i is kept in every layer (it is nonzero in the printed table).
"""
from __future__ import annotations

import math

import numpy as np

LN2 = math.log(2.0)


def mlsp2_scalar(x, theta, dtype=np.float64):
    """Scalar recursion on an array of layer-0 inputs x; returns A_n + x_n.
    ``dtype=np.float32`` evaluates every operation in FP32 from FP32-rounded
    inputs and coefficients (the scalar FP32 floor)."""
    x = np.asarray(x, dtype=dtype).copy()
    A = np.zeros_like(x)
    for a, b, c, d in theta:
        a, b, c, d = dtype(a), dtype(b), dtype(c), dtype(d)
        A = A + d * x
        x = a * x * x + b * x + c
    return (A + x).astype(np.float64)


def mlsp2_scalar_layers(x, theta):
    """Same recursion, returning the list of layer inputs x_0..x_n and A_n."""
    xs = [np.asarray(x, dtype=np.float64).copy()]
    A = np.zeros_like(xs[0])
    for a, b, c, d in theta:
        A = A + d * xs[-1]
        xs.append(a * xs[-1] * xs[-1] + b * xs[-1] + c)
    return xs, A


def mlsp2_matrix(X0: np.ndarray, theta) -> np.ndarray:
    """Matrix recursion of Alg. 2 (density part) in FP64:
    A_D <- A_D + d X ; X <- a X X + b X + c I ; returns A_D + X."""
    X = np.array(X0, dtype=np.float64)
    n = X.shape[0]
    I = np.eye(n)
    A = np.zeros_like(X)
    for a, b, c, d in theta:
        A = A + d * X
        X = a * (X @ X) + b * X + c * I
    return A + X


def entropy_input(x, alpha: float, mu0: float):
    """Layer-0 input of the entropy expansion, x0 = alpha (x - mu) + mu with the
    normalised chemical potential mu = mu0 (Eq. entropy expansion).  Reading of
    Alg. 2's "Y = alpha X + (1 - alpha) mu I": the mu there is the normalised
    mu0 of the model frame, which is what Eq. entropy expansion states."""
    return alpha * (np.asarray(x, dtype=np.float64) - mu0) + mu0


def entropy_scalar(x, theta, alpha: float, mu0: float, dtype=np.float64):
    """s~(x) = 4 ln2 F (1 - F), F = A_n + x_n of the recursion started at
    x0 = alpha (x - mu0) + mu0 (Eqs. entropy expansion, entropy expansion-s)."""
    F = mlsp2_scalar(entropy_input(x, alpha, mu0), theta, dtype=dtype)
    return 4.0 * LN2 * F * (1.0 - F)


def entropy_matrix(X0: np.ndarray, theta, alpha: float, mu0: float) -> float:
    """Matrix entropy of Alg. 2: Y0 = alpha (X0 - mu0 I) + mu0 I, the recursion
    with the entropy table, F = A_S + Y, S = 4 ln2 (Tr F - Tr F^2).

    Reading: Alg. 2 prints S = 4 ln2 (Tr(Y^2) - Tr(Y)), the negative of the
    trace of Eq. entropy expansion-s, 4 ln2 F (1 - F), which is >= 0 on [0, 1]
    like s itself (Eq. entropy); the sign of Eq. entropy expansion-s is taken."""
    n = X0.shape[0]
    Y0 = alpha * (np.array(X0, dtype=np.float64) - mu0 * np.eye(n)) + mu0 * np.eye(n)
    F = mlsp2_matrix(Y0, theta)
    return float(4.0 * LN2 * (np.trace(F) - np.trace(F @ F)))


def ansatz_entropy_of_t(t, alpha: float):
    """The alpha-rescaled m = 1 ansatz (Sec. II B): with the exact Fermi
    function f, s(t) ~ 4 ln2 f(alpha t) (1 - f(alpha t)), t = beta (x - mu)."""
    u = alpha * np.asarray(t, dtype=np.float64)
    f = 0.5 * (1.0 + np.tanh(-0.5 * u))
    return 4.0 * LN2 * f * (1.0 - f)


ALPHA_CURVATURE = 1.0 / math.sqrt(2.0 * LN2)   # s''(mu) exact (Sec. II B)
ALPHA_MINMAX = 0.842704                          # global max-error optimum (Sec. II B)
