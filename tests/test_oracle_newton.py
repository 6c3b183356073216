"""Pins of the oracle's Newton-Raphson solve for the chemical potential
(Sec. III A 4, Eqs. g, dg, delta_mu with the sign of Eq. drho taken from the
definition of D): the derivative against finite differences of the exact
Fermi operator, convergence to the root found by bisection, quadratic
convergence, agreement with the exact Fermi root within the model error, the
step limit, and a planted sign error that the checks catch."""
import math

import numpy as np

import workloads as wl
from oracle import fermi, newton, pipeline, rescale, tables

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
KT = 0.1


def chain(n=64, seed=3):
    return wl.chain_1d(n, seed)


def test_derivative_of_electron_count_matches_logistic_relation():
    # d/dmu sum_i f(eps_i; mu) by central differences = beta sum f (1 - f)
    # = beta (Tr D - Tr D^2) > 0: the sign the solver uses, from Eq. FD_Func
    H = chain()
    eps = np.linalg.eigvalsh(H)
    mu, h = 0.13, 1e-6
    fd = (np.sum(fermi.fermi(eps, mu + h, KT)) - np.sum(fermi.fermi(eps, mu - h, KT))) / (2 * h)
    f = fermi.fermi(eps, mu, KT)
    D, _, _, _ = fermi.eig_reference(H, mu, KT)
    closed = (np.trace(D) - np.sum(D * D)) / KT
    assert fd > 0
    assert abs(fd - np.sum(f * (1 - f)) / KT) < 1e-6 * fd
    assert abs(fd - closed) < 1e-6 * fd


def test_newton_converges_to_bisection_root_quadratically():
    H = chain()
    n = H.shape[0]
    n_occ = 30.0
    eps = np.linalg.eigvalsh(H)
    mu_star = newton.method_mu_bisection(H, n_occ, KT, [PRINTED], eps.min(), eps.max(), iters=80)
    assert abs(newton.method_electron_count(H, mu_star, KT, [PRINTED]) - n_occ) < 1e-8
    mu0 = mu_star + 3 * KT
    mu, hist, r = newton.newton_mu(H, n_occ, mu0, KT, [PRINTED], iterations=8, tol=1e-12)
    assert abs(mu - mu_star) < 1e-10
    assert abs(r["trD"] - n_occ) < 1e-9
    errs = [abs(h[0] - mu_star) for h in hist] + [abs(mu - mu_star)]
    # quadratic once close: e_{k+1} <= C e_k^2 with a modest C
    close = [(a, b) for a, b in zip(errs[:-1], errs[1:]) if 1e-7 < a < 1e-2]
    assert close, errs
    for a, b in close:
        assert b <= 50.0 * a * a + 1e-13, errs
    assert n > n_occ


def test_newton_root_agrees_with_exact_fermi_root():
    # the method's root differs from the exact one only by the fit error of the
    # printed table (2.2e-8 in f): |delta mu| <= n * 2.3e-8 / (beta Tr(D - D^2))
    H = chain(96, 5)
    n = H.shape[0]
    eps = np.linalg.eigvalsh(H)
    n_occ = 41.0
    mu_exact = fermi.mu_at_filling(eps, KT, n_occ)
    mu, hist, r = newton.newton_mu(H, n_occ, mu_exact - 2 * KT, KT, [PRINTED], iterations=10, tol=1e-12)
    f = fermi.fermi(eps, mu_exact, KT)
    slope = np.sum(f * (1 - f)) / KT
    assert abs(mu - mu_exact) <= n * 2.3e-8 / slope + 1e-12


def test_converged_instance_is_left_unchanged():
    assert newton.newton_step(10.0, 10.0 + 1e-9, 9.0, KT, 4.0, tol=1e-6) == 0.0
    # undefined step (D idempotent): no move
    assert newton.newton_step(10.0, 9.0, 9.0, KT, 4.0, tol=1e-6) == 0.0


def test_step_limited_to_a_sixteenth_of_the_width():
    H = chain()
    lo, hi = rescale.gershgorin(H)
    W = hi - lo
    r = pipeline.method_exact(H, lo + 0.3 * W, KT, [PRINTED])
    d = newton.newton_step(63.5, r["trD"], r["frobD"], KT, W, tol=1e-9)
    assert abs(d) <= W / 16 + 1e-15
    assert d > 0                                  # more electrons wanted -> mu up


def test_planted_sign_error_is_caught():
    # the printed sign of Eq. delta_mu moves mu away from the root: the
    # electron-count error grows after one step
    H = chain()
    n_occ = 30.0
    eps = np.linalg.eigvalsh(H)
    mu_star = newton.method_mu_bisection(H, n_occ, KT, [PRINTED], eps.min(), eps.max(), iters=80)
    mu0 = mu_star + 0.5 * KT
    r0 = pipeline.method_exact(H, mu0, KT, [PRINTED])
    W = newton.gershgorin_width(H)
    good = newton.newton_step(n_occ, r0["trD"], r0["frobD"], KT, W, tol=0.0)
    bad = -good                                   # the printed sign
    e0 = abs(r0["trD"] - n_occ)
    e_good = abs(newton.method_electron_count(H, mu0 + good, KT, [PRINTED]) - n_occ)
    e_bad = abs(newton.method_electron_count(H, mu0 + bad, KT, [PRINTED]) - n_occ)
    assert e_good < 0.1 * e0
    assert e_bad > e0
    assert math.isfinite(e_bad)
