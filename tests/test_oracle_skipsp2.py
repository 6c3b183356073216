"""Pins of the oracle's Skip-SP2 with one stored layer and one accumulator:
the Appendix's embedding of Eq. mlsp2 (evaluated against the Eq. mlsp2
recursion, on the printed table), the reduction to the one-term form at
beta = 0, closed forms of one- and two-layer tables with accumulator feedback,
the reverse-mode Jacobian against central differences, the matrix recursion
against the eigendecomposition, and the golden table's recorded fit."""
import json
import os

import numpy as np
import pytest

from oracle import altform, mlsp2, skipsp2, tables, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_embedding_of_the_printed_table():
    # Appendix embedding (beta = 0, initial accumulator A_0): same function
    x = np.linspace(0.0, 1.0, 20001)
    th = np.array(tables.PRINTED_B1500)
    tab = skipsp2.from_mlsp2(th)
    assert np.all(tab[:-1, 2] == 0.0)
    ref = mlsp2.mlsp2_scalar(x, th)
    assert np.max(np.abs(skipsp2.skip_scalar(x, tab) - ref)) < 1e-12
    # and on random tables with layers of both signs of a
    rng = np.random.default_rng(2)
    for L in (1, 2, 7):
        th = rng.normal(size=(L, 4)) * 0.5
        th[:, 0] = np.where(np.abs(th[:, 0]) < 0.2, 0.7, th[:, 0])
        xs = rng.uniform(0.0, 1.0, 200)
        ref = mlsp2.mlsp2_scalar(xs, th)
        got = skipsp2.skip_scalar(xs, skipsp2.from_mlsp2(th))
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), L


def test_no_feedback_is_the_one_term_form():
    # beta = 0, alpha = 1: u = delta + x, x' = u^2, A += gamma x; output A + x
    rng = np.random.default_rng(4)
    L = 9
    alt = rng.normal(size=(L + 1, 2)) * 0.3
    alt[L] = (0.0, 1.0)
    tab = np.zeros((L + 1, 4))
    tab[:L, 0] = alt[:L, 0]
    tab[:L, 1] = 1.0
    tab[:L, 3] = alt[:L, 1]
    tab[L, :2] = (0.0, 1.0)
    x = rng.uniform(0.0, 1.0, 300)
    assert np.max(np.abs(skipsp2.skip_scalar(x, tab) - altform.alt_scalar(x, alt))) < 1e-13


def test_closed_forms_with_feedback():
    x = np.linspace(0.0, 1.0, 101)
    d0, a0, b0, g0 = 0.3, -1.2, 0.7, 0.25
    A0, gL = -0.4, 1.3
    tab = np.array([[d0, a0, b0, g0], [A0, gL, 0.0, 0.0]])
    x1 = (d0 + a0 * x + b0 * A0) ** 2
    assert np.max(np.abs(skipsp2.skip_scalar(x, tab) - (A0 + g0 * x + gL * x1))) < 1e-14
    d1, a1, b1, g1 = -0.1, 0.9, -0.6, 0.5
    tab2 = np.array([[d0, a0, b0, g0], [d1, a1, b1, g1], [A0, gL, 0.0, 0.0]])
    A1 = A0 + g0 * x
    x2 = (d1 + a1 * x1 + b1 * A1) ** 2
    ref = A1 + g1 * x1 + gL * x2
    assert np.max(np.abs(skipsp2.skip_scalar(x, tab2) - ref)) < 1e-14


def test_jacobian_against_central_differences():
    rng = np.random.default_rng(7)
    L = 5
    tab = rng.normal(size=(L + 1, 4)) * 0.3
    tab[L, 2:] = 0.0
    x = rng.uniform(0.0, 1.0, 64)
    p = np.concatenate([tab[:L].ravel(), tab[L, :2]])

    def unflat(q):
        t = np.zeros((L + 1, 4))
        t[:L] = q[:4 * L].reshape(L, 4)
        t[L, :2] = q[4 * L:]
        return t

    for kind in ("fermi", "entropy"):
        F, J = skipsp2.forward_jacobian(tab, x, kind, alpha=0.8, mu0=0.4)
        assert J.shape == (64, 4 * L + 2)
        assert np.allclose(F, skipsp2.forward(tab, x, kind, alpha=0.8, mu0=0.4), atol=1e-14)
        h = 1e-6
        Jn = np.empty_like(J)
        for k in range(p.size):
            e = np.zeros(p.size)
            e[k] = h
            Jn[:, k] = (skipsp2.forward(unflat(p + e), x, kind, 0.8, 0.4)
                        - skipsp2.forward(unflat(p - e), x, kind, 0.8, 0.4)) / (2 * h)
        assert np.max(np.abs(J - Jn)) <= 1e-7 * max(1.0, np.max(np.abs(J))), kind


def test_matrix_recursion_on_eigenvalues():
    rng = np.random.default_rng(9)
    n = 11
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = rng.uniform(0.0, 1.0, n)
    tab = rng.normal(size=(5, 4)) * 0.4
    tab[4, 2:] = 0.0
    M = skipsp2.skip_matrix((Q * lam) @ Q.T, tab)
    assert np.max(np.abs(M - (Q * skipsp2.skip_scalar(lam, tab)) @ Q.T)) < 1e-12


def test_lm_fit_lowers_the_cost():
    beta0, mu0, L = 40.0, 1.0 / 3.0, 8
    x = train.sample_grid(3000, beta0, mu0)
    t0 = skipsp2.from_mlsp2(train.init_from_sp2(L, beta0, mu0))
    tab, hist = skipsp2.lm_fit(t0, x, "fermi", beta0, mu0, iters=30, accel=True)
    costs = [h[0] for h in hist]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 1e-3 * (0.5 * np.sum((skipsp2.forward(t0, x) - train.target(x, "fermi", beta0, mu0)) ** 2))


def test_golden_skip_table():
    # written by tests/golden/make_skip_table.py (oracle only)
    with open(os.path.join(ROOT, "tests", "golden", "skip_table.json")) as f:
        d = json.load(f)
    tab = np.array(d["skip"])
    assert tab.shape == (d["L"] + 1, 4)
    err = skipsp2.max_error(tab, "fermi", d["beta0"], d["mu0"], grid=200_001)
    assert abs(err - d["max_err"]) <= 1e-3 * d["max_err"] + 1e-15
    assert err < d["bound"]
    assert d["max_abs_beta"] > 0.0          # the accumulator feedback is used
    ent = np.array(d["skip_entropy"])
    e_err = skipsp2.max_error(ent, "entropy", d["beta0"], d["mu0"], alpha=d["alpha"], grid=200_001)
    assert abs(e_err - d["max_err_entropy"]) <= 1e-3 * d["max_err_entropy"] + 1e-15
