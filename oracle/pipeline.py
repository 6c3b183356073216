"""Alg. 2 end to end on one Hamiltonian, and the method-exact references
(TEST INFRASTRUCTURE ONLY).

``density_entropy`` takes Alg. 2's steps in order with plain FP64 matrix
products.  ``method_exact`` evaluates the same scalar recursion on the
eigenvalues of H and rebuilds the matrices from the eigenvectors: it isolates
the rounding error of an implementation (compare to it) from the model's fit
error (compare to ``fermi.eig_reference``).
"""
from __future__ import annotations

import math

import numpy as np

from . import fermi, mlsp2, rescale

LN2 = math.log(2.0)


def density_entropy(H: np.ndarray, mu: float, kT: float, tables, clamp: bool = False,
                    want_entropy: bool = True):
    """Returns dict(D, S, trD, frobD, rec).  D = A_D + X, or I - (A_D + X) when
    flipped (Appendix A); S per Alg. 2 with the sign of Eq. entropy expansion-s,
    using the table's entropy coefficients or, if it has none, its Fermi
    coefficients (theta_fermi strategy, Sec. II B).  S is returned in model
    units of Eq. entropy: sum over states of s, per spin, in k_B."""
    H0, rec = rescale.rescale(H, mu, kT, tables, clamp=clamp)
    if H0 is None:
        return dict(D=None, S=None, trD=None, frobD=None, rec=rec)
    t = tables[rec.model]
    n = H.shape[0]
    I = np.eye(n)
    F = mlsp2.mlsp2_matrix(H0, t.theta)
    D = I - F if rec.flip else F
    S = None
    if want_entropy:
        th = t.theta_entropy if t.theta_entropy is not None else t.theta
        S = mlsp2.entropy_matrix(H0, th, t.alpha, t.mu0)
    return dict(D=D, S=S, trD=float(np.trace(D)), frobD=float(np.sum(D * D)), rec=rec)


def method_exact(H: np.ndarray, mu: float, kT: float, tables, clamp: bool = False, lanczos: bool = False,
                 min_layers: bool = False):
    """D_rec = V diag(P(x0(eps))) V^T (flipped if needed) and
    S_rec = sum_i s~(x0(eps_i)), with P the FP64 scalar recursion.  ``lanczos``
    selects the Lanczos-tightened spectral bounds (oracle.lanczos),
    ``min_layers`` the fewest-layers model policy (rescale.select_model)."""
    H0, rec = rescale.rescale(H, mu, kT, tables, clamp=clamp, lanczos=lanczos, min_layers=min_layers)
    if H0 is None:
        return dict(D=None, S=None, rec=rec)
    t = tables[rec.model]
    eps, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    x0 = rescale.x0_of_eigenvalue(eps, mu, kT, rec, t)
    p = mlsp2.mlsp2_scalar(x0, t.theta)
    if rec.flip:
        p = 1.0 - p
    D = (V * p[None, :]) @ V.T
    th = t.theta_entropy if t.theta_entropy is not None else t.theta
    s = mlsp2.entropy_scalar(x0, th, t.alpha, t.mu0)
    return dict(D=D, S=float(np.sum(s)), trD=float(np.sum(p)), frobD=float(np.sum(p * p)),
                rec=rec, x0=x0, eps=eps)


def scalar_fp32_floor(H: np.ndarray, mu: float, kT: float, tables):
    """Per-eigenvalue difference between the scalar recursion evaluated in FP32
    and in FP64 on this H's mapped eigenvalues: the floor any FP32-class
    implementation of the same table faces (max over eigenvalues)."""
    r = method_exact(H, mu, kT, tables)
    t = tables[r["rec"].model]
    p64 = mlsp2.mlsp2_scalar(r["x0"], t.theta)
    p32 = mlsp2.mlsp2_scalar(r["x0"], t.theta, dtype=np.float32)
    return float(np.max(np.abs(p64 - p32)))
