"""Pins of the oracle's Lanczos spectral bounds: the counter-based start
vector against the generator's published first outputs, the recurrence
against its defining properties (orthonormal basis, T = V^T H V, Cauchy
interlacing, exact spectrum after n steps), and the bounds against the
eigenvalues of every workload family (enclosure, tighter than Gershgorin)."""
import numpy as np
import pytest

import workloads as wl
from oracle import lanczos, rescale


def test_splitmix64_published_first_outputs():
    # a generator seeded with 0 returns these two values first
    assert lanczos.splitmix64(0) == 0xE220A8397B1DCDAF
    assert lanczos.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_start_vector_is_unit_and_spread():
    q = lanczos.start_vector(1000)
    assert abs(np.linalg.norm(q) - 1.0) < 1e-14
    # values 2u - 1 are spread over (-1, 1): mean near 0, second moment near 1/3 before scaling
    raw = q * np.linalg.norm([2.0 * ((lanczos.splitmix64(i) >> 11) * 2.0 ** -53) - 1.0 for i in range(1000)])
    assert abs(raw.mean()) < 0.05 and abs(np.mean(raw ** 2) - 1 / 3) < 0.05


def _basis(H, k):
    # the Lanczos vectors rebuilt with full re-orthogonalisation, for comparison
    n = H.shape[0]
    V = np.zeros((n, k))
    V[:, 0] = lanczos.start_vector(n)
    for j in range(1, k):
        w = H @ V[:, j - 1]
        w -= V[:, :j] @ (V[:, :j].T @ w)
        w -= V[:, :j] @ (V[:, :j].T @ w)
        V[:, j] = w / np.linalg.norm(w)
    return V


def test_tridiagonal_is_projection_of_H():
    H = wl.chain_1d(120, 2)
    k = 8
    a, b = lanczos.lanczos_tridiagonal(H, k)
    V = _basis(H, k)
    T = V.T @ H @ V
    assert np.allclose(np.diag(T), a, atol=1e-10)
    assert np.allclose(np.abs(np.diag(T, 1)), b[:-1], atol=1e-10)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-12)


def test_interlacing_and_exact_after_n_steps():
    rng = np.random.default_rng(4)
    lam = np.sort(rng.uniform(-3, 5, 12))
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    H = (Q * lam) @ Q.T
    a, b = lanczos.lanczos_tridiagonal(H, 5)
    t_lo, _, t_hi, _ = lanczos.ritz_extremes(a, b)
    assert lam[0] - 1e-12 <= t_lo and t_hi <= lam[-1] + 1e-12          # Cauchy interlacing
    a, b = lanczos.lanczos_tridiagonal(H, 12)
    t_lo, r_lo, t_hi, r_hi = lanczos.ritz_extremes(a, b)
    assert abs(t_lo - lam[0]) < 1e-9 and abs(t_hi - lam[-1]) < 1e-9      # n steps: exact
    # residual bound: an eigenvalue lies within r of each Ritz value
    a, b = lanczos.lanczos_tridiagonal(H, 6)
    t_lo, r_lo, t_hi, r_hi = lanczos.ritz_extremes(a, b)
    assert np.min(np.abs(lam - t_lo)) <= r_lo + 1e-12
    assert np.min(np.abs(lam - t_hi)) <= r_hi + 1e-12


def test_scalar_matrix_keeps_degenerate_bounds():
    H = 0.7 * np.eye(40)
    assert lanczos.bounds(H) == (0.7, 0.7)


def _families():
    out = [("chain256", wl.chain_1d(256, 0)), ("chain97", wl.chain_1d(97, 5)),
           ("lattice512", wl.lattice_3d((8, 8, 8), 0)), ("lattice1024", wl.lattice_3d((8, 8, 16), 1)),
           ("lattice_lr1024", wl.lattice_3d((8, 8, 16), 2, longrange_frac=0.05, longrange_sigma=0.05))]
    for b in wl.ragged_batch(10, 3):
        out.append(("rot%d" % b["n"], b["H"]))
    return out


@pytest.mark.parametrize("name,H", _families(), ids=lambda x: x if isinstance(x, str) else "")
def test_bounds_enclose_spectrum_and_beat_gershgorin(name, H):
    ev = np.linalg.eigvalsh(H)
    lo, hi = lanczos.bounds(H)
    g_lo, g_hi = rescale.gershgorin(H)
    assert lo <= ev[0] and hi >= ev[-1], (name, lo - ev[0], hi - ev[-1])
    assert g_lo <= lo and hi <= g_hi
    # the noise (lattices, chains) and the dense rotation make Gershgorin loose
    assert (hi - lo) < 0.8 * (g_hi - g_lo), name
