"""Seeded synthetic Hamiltonians shared by the tests, the oracle scripts and the bench.

This module only draws random numbers and assembles matrices; it holds none of
the Fermi-operator method's arithmetic (no spectral bounds, no rescaling, no
recursion, no Fermi function).  Every generator takes an explicit seed and uses
``numpy.random.default_rng(seed)`` so both sides of a parity test see identical
FP64 inputs.

Workload recipes (units: eV, k_B absorbed so beta = 1/kT):

* ``chain_1d``      -- open 1D tight-binding chain: on-site U(-1,1), nearest-
  neighbour hopping -1, plus symmetrised dense noise 0.01*(G+G^T)/2, G~N(0,1).
* ``lattice_3d``    -- the same on an open nx*ny*nz cubic lattice (6-neighbour
  hopping); optionally a fraction of random long-range couplings N(0, sigma)
  on upper-triangle pairs, mirrored.
* ``rotated_spectrum`` -- H = Q diag(lam) Q^T, lam ~ U(lo, hi), Q Haar-random
  (QR of a Gaussian matrix with the sign of R's diagonal folded into Q).
* ``ragged_batch``  -- many rotated-spectrum instances with n ~ U{nmin..nmax},
  kT ~ U(kT_lo, kT_hi), mu ~ U(mu_lo, mu_hi).
* ``appendix_matrix`` -- the paper's random test matrix (Appendix A harness):
  U(0,1) entries, then H + H^T.
"""
from __future__ import annotations

import numpy as np


def chain_1d(n: int, seed: int, noise: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    H = np.zeros((n, n))
    H[np.arange(n), np.arange(n)] = rng.uniform(-1.0, 1.0, n)
    i = np.arange(n - 1)
    H[i, i + 1] = -1.0
    H[i + 1, i] = -1.0
    G = rng.standard_normal((n, n))
    H += noise * (G + G.T) / 2.0
    return H


def lattice_3d(dims, seed: int, noise: float = 0.01, longrange_frac: float = 0.0,
               longrange_sigma: float = 0.0) -> np.ndarray:
    nx, ny, nz = dims
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    H = np.zeros((n, n))
    H[np.arange(n), np.arange(n)] = rng.uniform(-1.0, 1.0, n)
    idx = np.arange(n).reshape(nx, ny, nz)
    for ax in range(3):
        a = np.take(idx, range(0, idx.shape[ax] - 1), axis=ax).ravel()
        b = np.take(idx, range(1, idx.shape[ax]), axis=ax).ravel()
        H[a, b] = -1.0
        H[b, a] = -1.0
    G = rng.standard_normal((n, n))
    H += noise * (G + G.T) / 2.0
    if longrange_frac > 0.0:
        iu, ju = np.triu_indices(n, 1)
        pick = rng.random(iu.size) < longrange_frac
        vals = rng.normal(0.0, longrange_sigma, int(pick.sum()))
        H[iu[pick], ju[pick]] += vals
        H[ju[pick], iu[pick]] += vals
    return H


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def rotated_spectrum(n: int, seed: int, lo: float = -10.0, hi: float = 10.0):
    """Returns (H, lam): H = Q diag(lam) Q^T with the drawn eigenvalues lam."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(lo, hi, n)
    Q = haar_orthogonal(n, rng)
    H = (Q * lam[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    return H, lam


def ragged_sizes(nb: int, seed: int, nmin: int = 64, nmax: int = 768):
    rng = np.random.default_rng(seed)
    return rng.integers(nmin, nmax + 1, nb)


def ragged_batch(nb: int, seed: int, nmin: int = 64, nmax: int = 768,
                 kT_lo: float = 0.02, kT_hi: float = 0.5, mu_lo: float = -5.0,
                 mu_hi: float = 5.0):
    """List of dicts {n, H, mu, kT, lam}; instance b uses seed (seed, b)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, nb)
    kTs = rng.uniform(kT_lo, kT_hi, nb)
    mus = rng.uniform(mu_lo, mu_hi, nb)
    out = []
    for b in range(nb):
        H, lam = rotated_spectrum(int(ns[b]), seed * 100003 + b)
        out.append(dict(n=int(ns[b]), H=H, mu=float(mus[b]), kT=float(kTs[b]), lam=lam))
    return out


def appendix_matrix(seed: int, n: int = 100) -> np.ndarray:
    rng = np.random.default_rng(seed=seed)
    H = rng.uniform(0.0, 1.0, (n, n))
    return H + H.T


def appendix_rng(seed: int) -> np.random.Generator:
    """Generator positioned after ``appendix_matrix`` drew its entries, so the
    harness can continue drawing beta and mu from the same stream."""
    rng = np.random.default_rng(seed=seed)
    rng.uniform(0.0, 1.0, (100, 100))
    return rng


def pack_batch(Hs):
    """Concatenate row-major FP64 matrices into one flat buffer; returns
    (flat, offsets) with offsets in elements."""
    offs = []
    o = 0
    for H in Hs:
        offs.append(o)
        o += H.shape[0] * H.shape[0]
    flat = np.empty(o, dtype=np.float64)
    for H, off in zip(Hs, offs):
        n = H.shape[0]
        flat[off:off + n * n] = np.ascontiguousarray(H).ravel()
    return flat, np.array(offs, dtype=np.int64)
