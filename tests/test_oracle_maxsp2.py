"""Pins of the oracle's Max-SP2 (Sec. II A 2, Eq. maxsp2) and of Skip-SP2
with k stored layers and K accumulators (Sec. II A 3): hand-expanded closed
forms of one- and two-layer tables, the Appendix's embeddings checked against
the already pinned Eq. mlsp2 and one-accumulator recursions, the embedding of
Skip-SP2 in Max-SP2 on random tables, the reverse-mode Jacobian and the
Skip-SP2 chain-rule Jacobian against central differences, the matrix
recursion against the eigendecomposition, the fits lowering their cost, the
density of a solve against the Eq. mlsp2 path, and the golden tables'
recorded fits."""
import json
import os

import numpy as np
import pytest

from oracle import maxsp2, mlsp2, skipsp2, tables, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _random_max(rng, L, scale=0.5):
    return rng.normal(size=maxsp2.nparams(L)) * scale


def _random_skip(rng, L, k, K, scale=0.4):
    return dict(alpha=rng.normal(size=(L, k + 1)) * scale, beta=rng.normal(size=(L, K)) * scale,
                gamma=rng.normal(size=(L, K)) * scale, A0=rng.normal(size=K) * scale, gL=float(rng.normal()))


def test_flat_layout_roundtrip_and_count():
    rng = np.random.default_rng(1)
    for L in (1, 2, 5, 20):
        p = _random_max(rng, L)
        assert p.size == L * (L + 5) // 2 + 2
        d, g, th, c = maxsp2.unflat(p, L)
        assert [t.size for t in th] == list(range(1, L + 1))
        assert np.array_equal(maxsp2.flat(d, g, th, c), p)


def test_closed_forms():
    x = np.linspace(-0.5, 1.5, 101)
    # one layer: f = c + g0 x + g1 (d + t x)^2, expanded by hand
    d, t, c, g0, g1 = 0.3, -1.7, 0.25, 0.6, -0.8
    p = np.array([d, g0, t, c, g1])
    ref = c + g0 * x + g1 * (d * d + 2.0 * d * t * x + t * t * x * x)
    assert np.max(np.abs(maxsp2.max_scalar(x, p, 1) - ref)) < 1e-14
    # two layers on integers: x1 = x^2, x2 = (x1 - 1)^2 = x^4 - 2 x^2 + 1, f = x2
    p2 = maxsp2.flat([0.0, -1.0], [0.0, 0.0, 1.0], [np.array([1.0]), np.array([0.0, 1.0])], 0.0)
    assert maxsp2.max_scalar(np.array([2.0]), p2, 2)[0] == 9.0
    assert np.max(np.abs(maxsp2.max_scalar(x, p2, 2) - (x ** 4 - 2 * x ** 2 + 1))) < 1e-14
    # two layers, both connections of layer 1 used:
    # u1 = d1 + t10 x + t11 (d0 + t00 x)^2
    d0, t00, d1, t10, t11 = 0.2, 0.9, -0.4, 0.7, -1.1
    gg = [0.1, -0.2, 0.5]
    p3 = maxsp2.flat([d0, d1], gg, [np.array([t00]), np.array([t10, t11])], 0.05)
    x1 = (d0 + t00 * x) ** 2
    x2 = (d1 + t10 * x + t11 * x1) ** 2
    assert np.max(np.abs(maxsp2.max_scalar(x, p3, 2) - (0.05 + gg[0] * x + gg[1] * x1 + gg[2] * x2))) < 1e-14


def test_skip_closed_form_two_stored_layers_two_accumulators():
    rng = np.random.default_rng(3)
    t = _random_skip(rng, 2, 2, 2)
    al, be, ga, A0, gL = t["alpha"], t["beta"], t["gamma"], t["A0"], t["gL"]
    x = rng.uniform(0.0, 1.0, 50)
    # layer 0 reads x_0 only (no x_{-1}); layer 1 reads x_1, x_0 and A_1
    x1 = (al[0, 2] + al[0, 0] * x + be[0, 0] * A0[0] + be[0, 1] * A0[1]) ** 2
    A1 = [A0[l] + ga[0, l] * x for l in range(2)]
    x2 = (al[1, 2] + al[1, 0] * x1 + al[1, 1] * x + be[1, 0] * A1[0] + be[1, 1] * A1[1]) ** 2
    A2 = [A1[l] + ga[1, l] * x1 for l in range(2)]
    ref = gL * x2 + A2[0] + A2[1]
    assert np.max(np.abs(maxsp2.skip_scalar(x, t) - ref)) < 1e-13


def test_mlsp2_embedding_printed_and_random():
    x = np.linspace(0.0, 1.0, 20001)
    th = np.array(tables.PRINTED_B1500)
    p = maxsp2.mlsp2_to_max(th)
    assert p.size == maxsp2.nparams(26)
    assert np.max(np.abs(maxsp2.max_scalar(x, p, 26) - mlsp2.mlsp2_scalar(x, th))) < 1e-12
    rng = np.random.default_rng(5)
    for L in (1, 3, 8):
        th = rng.normal(size=(L, 4)) * 0.5
        th[:, 0] = np.where(np.abs(th[:, 0]) < 0.2, 0.7, th[:, 0])
        xs = rng.uniform(0.0, 1.0, 200)
        ref = mlsp2.mlsp2_scalar(xs, th)
        got = maxsp2.max_scalar(xs, maxsp2.mlsp2_to_max(th), L)
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), L


def test_one_accumulator_skip_in_max_with_feedback():
    rng = np.random.default_rng(6)
    for L in (1, 4, 9):
        tab = rng.normal(size=(L + 1, 4)) * 0.4
        tab[L, 2:] = 0.0
        x = rng.uniform(0.0, 1.0, 100)
        ref = skipsp2.skip_scalar(x, tab)
        assert np.max(np.abs(maxsp2.max_scalar(x, maxsp2.skip1_to_max(tab), L) - ref)) < 1e-13
        # and through the general (k, K) form with the extra connections unused
        for k, K in ((1, 1), (2, 2), (3, 1)):
            g = maxsp2.skip_from_skip1(tab, k, K, beta_extra=0.3)
            assert np.max(np.abs(maxsp2.skip_scalar(x, g) - ref)) < 1e-13, (L, k, K)


@pytest.mark.parametrize("k,K", [(1, 1), (2, 2), (3, 1), (1, 3), (2, 0)])
def test_skip_in_max_on_random_tables(k, K):
    rng = np.random.default_rng(10 * k + K)
    for L in (1, 2, 6):
        t = _random_skip(rng, L, k, K)
        x = rng.uniform(0.0, 1.0, 150)
        ref = maxsp2.skip_scalar(x, t)
        got = maxsp2.max_scalar(x, maxsp2.skip_to_max(t), L)
        assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), L
    # with k >= L every earlier layer is a stored one: theta = alpha reversed
    t = _random_skip(rng, 3, 3, K)
    if K == 0:
        d, g, th, c = maxsp2.unflat(maxsp2.skip_to_max(t), 3)
        for i in range(3):
            assert np.allclose(th[i], t["alpha"][i, i::-1])


def test_max_jacobian_against_central_differences():
    rng = np.random.default_rng(11)
    L = 4
    p = _random_max(rng, L, 0.4)
    x = rng.uniform(0.0, 1.0, 64)
    for kind in ("fermi", "entropy"):
        F, J = maxsp2.forward_jacobian(p, L, x, kind, alpha=0.8, mu0=0.4)
        assert J.shape == (64, maxsp2.nparams(L))
        assert np.allclose(F, maxsp2.forward(p, L, x, kind, alpha=0.8, mu0=0.4), atol=1e-14)
        h = 1e-6
        Jn = np.empty_like(J)
        for m in range(p.size):
            e = np.zeros(p.size)
            e[m] = h
            Jn[:, m] = (maxsp2.forward(p + e, L, x, kind, 0.8, 0.4) - maxsp2.forward(p - e, L, x, kind, 0.8, 0.4)) / (2 * h)
        assert np.max(np.abs(J - Jn)) <= 1e-7 * max(1.0, np.max(np.abs(J))), kind


def test_skip_chain_rule_jacobian_against_central_differences():
    rng = np.random.default_rng(12)
    L, k, K = 4, 2, 2
    t = _random_skip(rng, L, k, K, 0.3)
    t["A0"][1:] = 0.0                    # the fit's parametrisation: one initial accumulator
    q = maxsp2.skip_pack(t)
    assert q.size == (1 + k + 2 * K) * L + 2
    x = rng.uniform(0.0, 1.0, 40)
    _, Jm = maxsp2.forward_jacobian(maxsp2.skip_to_max(t), L, x)
    J = Jm @ maxsp2.skip_embedding_jacobian(q, L, k, K)
    h = 1e-6
    Jn = np.empty_like(J)
    for m in range(q.size):
        e = np.zeros(q.size)
        e[m] = h
        Jn[:, m] = (maxsp2.skip_scalar(x, maxsp2.skip_unpack(q + e, L, k, K))
                    - maxsp2.skip_scalar(x, maxsp2.skip_unpack(q - e, L, k, K))) / (2 * h)
    assert np.max(np.abs(J - Jn)) <= 1e-7 * max(1.0, np.max(np.abs(J)))


def test_matrix_recursions_on_eigenvalues():
    rng = np.random.default_rng(13)
    n = 11
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = rng.uniform(0.0, 1.0, n)
    X = (Q * lam) @ Q.T
    p = _random_max(rng, 5, 0.4)
    assert np.max(np.abs(maxsp2.max_matrix(X, p, 5) - (Q * maxsp2.max_scalar(lam, p, 5)) @ Q.T)) < 1e-11
    t = _random_skip(rng, 5, 2, 2)
    assert np.max(np.abs(maxsp2.skip_matrix(X, t) - (Q * maxsp2.skip_scalar(lam, t)) @ Q.T)) < 1e-11


def test_fits_lower_the_cost():
    beta0, mu0, L = 40.0, 1.0 / 3.0, 6
    x = train.sample_grid(3000, beta0, mu0)
    y = train.target(x, "fermi", beta0, mu0)
    th0 = train.init_from_sp2(L, beta0, mu0)
    p0 = maxsp2.mlsp2_to_max(th0)
    p, hist = maxsp2.lm_fit(p0, L, x, "fermi", beta0, mu0, iters=25, accel=True)
    costs = [h[0] for h in hist]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 1e-2 * 0.5 * np.sum((maxsp2.max_scalar(x, p0, L) - y) ** 2)
    t0 = maxsp2.skip_from_skip1(skipsp2.from_mlsp2(th0), 2, 2, beta_extra=0.01)
    t, hist = maxsp2.skip_lm_fit(t0, "fermi", x, beta0, mu0, iters=40, accel=True)
    costs = [h[0] for h in hist]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 0.05 * 0.5 * np.sum((maxsp2.skip_scalar(x, t0) - y) ** 2)
    assert np.max(np.abs(t["beta"][:, 1])) > 0.0 and np.max(np.abs(t["gamma"][:, 1])) > 0.0


def test_method_exact_matches_the_mlsp2_path():
    # the embedded printed table gives the density of the one-accumulator path
    rng = np.random.default_rng(14)
    n = 40
    A = rng.normal(size=(n, n)) * 0.3
    H = 0.5 * (A + A.T)
    th = np.array(tables.PRINTED_B1500)
    the = np.array(tables.THETA_FERMI_ENTROPY) if hasattr(tables, "THETA_FERMI_ENTROPY") else th
    ref = skipsp2.method_exact(H, 0.1, 0.02, skipsp2.from_mlsp2(th), 1500.0, 1.0 / 3.0, 0.842704,
                               skipsp2.from_mlsp2(the))
    got = maxsp2.method_exact(H, 0.1, 0.02, maxsp2.mlsp2_to_max(th), 26, 1500.0, 1.0 / 3.0, 0.842704,
                              maxsp2.mlsp2_to_max(the), the.shape[0])
    assert np.max(np.abs(got["D"] - ref["D"])) < 1e-10
    assert abs(got["S"] - ref["S"]) < 1e-8 * max(1.0, abs(ref["S"]))


def test_golden_max_table():
    # written by tests/golden/make_max_table.py (oracle only)
    with open(os.path.join(ROOT, "tests", "golden", "max_table.json")) as f:
        d = json.load(f)
    L = d["L"]
    p = np.array(d["max"])
    assert p.size == maxsp2.nparams(L)
    err = maxsp2.max_error(p, L, "fermi", d["beta0"], d["mu0"], grid=200_001)
    assert abs(err - d["max_err"]) <= 1e-3 * d["max_err"] + 1e-15
    pe = np.array(d["max_entropy"])
    e_err = maxsp2.max_error(pe, L, "entropy", d["beta0"], d["mu0"], alpha=d["alpha"], grid=200_001)
    assert abs(e_err - d["max_err_entropy"]) <= 1e-3 * d["max_err_entropy"] + 1e-15
    t = {k: np.array(v) if isinstance(v, list) else v for k, v in d["skip22"].items()}
    assert t["alpha"].shape == (L, 3) and t["beta"].shape == (L, 2)
    s_err = maxsp2.max_error(maxsp2.skip_to_max(t), L, "fermi", d["beta0"], d["mu0"], grid=200_001)
    assert abs(s_err - d["skip22_max_err"]) <= 1e-3 * d["skip22_max_err"] + 1e-15
    # the second stored layer and the second accumulator are used
    assert np.max(np.abs(t["alpha"][:, 1])) > 1e-3 and np.max(np.abs(t["gamma"][:, 1])) > 1e-3
    # a 12-layer Eq. mlsp2 start embedded in either family is far worse than the fits
    th0 = train.init_from_sp2(L, d["beta0"], d["mu0"])
    assert maxsp2.max_error(maxsp2.mlsp2_to_max(th0), L, "fermi", d["beta0"], d["mu0"], grid=20_001) > 100 * err
