"""Thin callers of the library's training entry points (a7; Sec. II C), used by
``train_tables``.  The sample set (ftsp2_train_samples), the starting tables
(ftsp2_train_init, ftsp2_train_init_alt, ftsp2_mlsp2_to_skip), the layer count
(ftsp2_layer_count) and the fit itself (ftsp2_train_coeffs and its one-term
and Skip-SP2 variants) are all computed inside the library; this module only
passes arguments and returns the results.
"""
from __future__ import annotations


def _ft():
    import paper_2605_08523_gb300 as ft
    return ft


def sample_points(N: int, beta0: float, mu0: float, seed: int = 0):
    """The library's training samples (ftsp2_train_samples)."""
    return _ft().ftsp2_train_samples(beta0, mu0, N, seed)


def sp2_init(L: int, beta0: float, mu0: float):
    """The library's starting Eq. mlsp2 table (ftsp2_train_init)."""
    return _ft().ftsp2_train_init(L, beta0, mu0)


def sp2_alt_init(L: int, mu0: float):
    """The library's starting table of the one-term form (ftsp2_train_init_alt)."""
    return _ft().ftsp2_train_init_alt(L, mu0)


def skip_from_mlsp2(theta):
    """Skip-SP2 embedding of Eq. mlsp2 rows (ftsp2_mlsp2_to_skip)."""
    return _ft().ftsp2_mlsp2_to_skip(theta)


def layer_count(beta_p: float) -> float:
    """Eq. layer count (ftsp2_layer_count)."""
    return _ft().ftsp2_layer_count(beta_p)


def train_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                nsamples: int = 100_000, theta_init=None, accel: bool = True, seed: int = 0):
    """Fit an Eq. mlsp2 table on the GPU (ftsp2_train_coeffs).  Returns (theta, report)."""
    return ft.ftsp2_train_coeffs(target, beta0, mu0, L=L, theta_init=theta_init, nsamples=nsamples, seed=seed,
                                 iterations=iterations, accel=accel, alpha=alpha)


def train_alt_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                    nsamples: int = 100_000, alt_init=None, accel: bool = True, seed: int = 0):
    """Fit a table of the one-term form on the GPU (ftsp2_train_coeffs_alt)."""
    return ft.ftsp2_train_coeffs_alt(target, beta0, mu0, L=L, alt_init=alt_init, nsamples=nsamples, seed=seed,
                                     iterations=iterations, accel=accel, alpha=alpha)


def train_skip_table(ft, target: int, beta0: float, mu0: float, L: int, alpha: float = 1.0, iterations: int = 500,
                     nsamples: int = 100_000, skip_init=None, accel: bool = True, seed: int = 0):
    """Fit a Skip-SP2 table on the GPU (ftsp2_train_coeffs_skip)."""
    return ft.ftsp2_train_coeffs_skip(target, beta0, mu0, L=L, skip_init=skip_init, nsamples=nsamples, seed=seed,
                                      iterations=iterations, accel=accel, alpha=alpha)
