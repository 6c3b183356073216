"""Fermi-Dirac occupation, electronic entropy and their matrix versions by
eigendecomposition (TEST INFRASTRUCTURE ONLY; see ``oracle/__init__``).

Units: energies in eV with k_B absorbed, beta = 1/kT.  The entropy is returned
per spin channel in units of k_B (reading of the "factor of 2 for spin" remark
next to Eq. entropy-matrix: the spin factor belongs to the caller, as in the
free energy G = 2 Tr[D(H - mu)] - 2 T S).
"""
from __future__ import annotations

import math

import numpy as np


def fermi(eps, mu: float, kT: float):
    """f(eps) = 1 / (exp((eps - mu)/kT) + 1)  (Eq. FD_Func), evaluated without
    overflow for large |eps - mu|/kT."""
    t = (np.asarray(eps, dtype=np.float64) - mu) / kT
    out = np.empty_like(t)
    pos = t > 0
    e = np.exp(-t[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(t[~pos]))
    return out


def entropy_of_t(t):
    """s as a function of t = (eps - mu)/kT, s = -f ln f - (1-f) ln(1-f)
    (Eq. entropy) with f = 1/(e^t + 1).  Written as
    ln(1 + e^-|t|) + |t| e^-|t| / (1 + e^-|t|), which is the same function
    (expand -f ln f - (1-f) ln(1-f) for t > 0 and use s(t) = s(-t)) and has no
    0 * log 0 at large |t|."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    e = np.exp(-a)
    return np.log1p(e) + a * e / (1.0 + e)


def entropy(eps, mu: float, kT: float):
    return entropy_of_t((np.asarray(eps, dtype=np.float64) - mu) / kT)


def entropy_of_f(f):
    """s(f) = -f ln f - (1-f) ln(1-f) with 0 ln 0 = 0 (Sec. II B)."""
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    m = (f > 0) & (f < 1)
    out[m] = -f[m] * np.log(f[m]) - (1 - f[m]) * np.log(1 - f[m])
    return out


def eig_reference(H: np.ndarray, mu: float, kT: float):
    """D_ref = V diag(f(eps)) V^T, S_ref = sum_i s(eps_i), Tr D_ref = sum_i f(eps_i)
    from an FP64 symmetric eigendecomposition (the plain definitions the method
    approximates: Eq. FD_Func and the matrix form below it, Eq. entropy-matrix)."""
    eps, V = np.linalg.eigh(H)
    f = fermi(eps, mu, kT)
    D = (V * f[None, :]) @ V.T
    S = float(np.sum(entropy(eps, mu, kT)))
    return D, S, float(np.sum(f)), eps


def matrix_function(H: np.ndarray, fn):
    """V diag(fn(eps)) V^T for a scalar function fn of the eigenvalues."""
    eps, V = np.linalg.eigh(H)
    return (V * fn(eps)[None, :]) @ V.T


def mu_at_filling(eps, kT: float, n_occ: float, iters: int = 200) -> float:
    """Chemical potential with sum_i f(eps_i) = n_occ (Sec. II A), by bisection
    on the eigenvalues.  Used to place mu at half filling (n_occ = n/2)."""
    eps = np.asarray(eps, dtype=np.float64)
    lo, hi = float(eps.min()) - 50.0 * kT - 1.0, float(eps.max()) + 50.0 * kT + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.sum(fermi(eps, mid, kT)) > n_occ:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def jacobi_eigh(A, sweeps: int = 60, tol: float = 1e-15):
    """Cyclic Jacobi eigenvalue algorithm in pure Python (tiny matrices only).
    Independent of LAPACK; used to cross-check ``numpy.linalg.eigh`` in the
    brute-force pins.  Returns (eigenvalues ascending, eigenvectors as columns)."""
    n = len(A)
    a = [[float(A[i][j]) for j in range(n)] for i in range(n)]
    v = [[1.0 if i == j else 0.0 for j in range(n)] for i in range(n)]
    for _ in range(sweeps):
        off = sum(a[i][j] ** 2 for i in range(n) for j in range(n) if i != j)
        if off < tol * tol:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(a[p][q]) < 1e-300:
                    continue
                theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q])
                t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                for k in range(n):
                    akp, akq = a[k][p], a[k][q]
                    a[k][p] = c * akp - s * akq
                    a[k][q] = s * akp + c * akq
                for k in range(n):
                    apk, aqk = a[p][k], a[q][k]
                    a[p][k] = c * apk - s * aqk
                    a[q][k] = s * apk + c * aqk
                for k in range(n):
                    vkp, vkq = v[k][p], v[k][q]
                    v[k][p] = c * vkp - s * vkq
                    v[k][q] = s * vkp + c * vkq
    w = [a[i][i] for i in range(n)]
    order = sorted(range(n), key=lambda i: w[i])
    return ([w[i] for i in order], [[v[r][i] for i in order] for r in range(n)])
