"""Pins of the oracle's one-term form (Eq. mlsp2_alt): the SP2 sequence it
represents exactly, the embedding into Eq. mlsp2 checked by evaluating the two
recursions independently, the chain-rule Jacobian against central
differences, the matrix recursion against the eigendecomposition, and the
library's host conversion (no GPU needed) against the oracle's."""
import json
import os

import numpy as np
import pytest

from oracle import altform, mlsp2, sp2, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def test_sp2_sequence_is_exact_in_the_one_term_form():
    # x^2 and 2x - x^2 = 1 - (1 - x)^2 are both squares of t + y with y = x or
    # 1 - x; the composition must match the plain SP2 polynomials
    x = np.linspace(0.0, 1.0, 1001)
    for mu_p, L in ((1.0 / 3.0, 26), (0.5, 12), (0.8, 9)):
        ref = mlsp2.mlsp2_scalar(x, sp2.sp2_table(mu_p, L))
        got = altform.alt_scalar(x, altform.sp2_alt(mu_p, L))
        assert np.max(np.abs(got - ref)) < 1e-13, (mu_p, L)
    # a hand-built four-layer table against its closed form:
    # y1 = x^2, y2 = (-1 + y1)^2, y3 = y2^2, y4 = (-1 + y3)^2, f = y4
    alt = np.zeros((5, 2))
    alt[1, 0] = -1.0
    alt[3, 0] = -1.0
    alt[4] = (0.0, 1.0)
    f = x * x
    y = (1.0 - f) ** 2
    y = y * y
    y = (y - 1.0) ** 2
    assert np.max(np.abs(altform.alt_scalar(x, alt) - y)) < 1e-14


def test_parameter_count():
    assert altform.sp2_alt(0.4, 17).shape == (18, 2)      # 2L + 2 parameters


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_embedding_into_mlsp2(seed):
    rng = np.random.default_rng(seed)
    L = 1 + seed * 5
    alt = rng.normal(size=(L + 1, 2)) * 0.4
    x = rng.uniform(0.0, 1.0, 500)
    th = altform.to_mlsp2(alt)
    assert th.shape == (L, 4)
    # every layer but the last has a = 1, b = 2 t, c = t^2 (a pure square)
    assert np.all(th[:-1, 0] == 1.0)
    ref = altform.alt_scalar(x, alt)
    assert np.max(np.abs(mlsp2.mlsp2_scalar(x, th) - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_jacobian_against_central_differences():
    rng = np.random.default_rng(5)
    alt = rng.normal(size=(7, 2)) * 0.3
    x = rng.uniform(0.0, 1.0, 64)
    for kind in ("fermi", "entropy"):
        F, J = altform.forward_jacobian(alt, x, kind, alpha=0.8, mu0=0.4)
        assert np.allclose(F, altform.forward(alt, x, kind, alpha=0.8, mu0=0.4), atol=1e-13)
        h = 1e-6
        Jn = np.empty_like(J)
        for k in range(alt.size):
            e = np.zeros(alt.size)
            e[k] = h
            e = e.reshape(alt.shape)
            Jn[:, k] = (altform.forward(alt + e, x, kind, 0.8, 0.4) - altform.forward(alt - e, x, kind, 0.8, 0.4)) / (2 * h)
        assert np.max(np.abs(J - Jn)) <= 1e-6 * max(1.0, np.max(np.abs(J))), kind


def test_matrix_recursion_is_the_scalar_one_on_eigenvalues():
    rng = np.random.default_rng(3)
    n = 12
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    lam = rng.uniform(0.0, 1.0, n)
    X0 = (Q * lam) @ Q.T
    alt = rng.normal(size=(6, 2)) * 0.3
    M = altform.alt_matrix(X0, alt)
    ref = (Q * altform.alt_scalar(lam, alt)) @ Q.T
    assert np.max(np.abs(M - ref)) < 1e-12
    # diagonal input: exact scalar recursion per entry
    D = altform.alt_matrix(np.diag(lam), alt)
    assert np.max(np.abs(np.diag(D) - altform.alt_scalar(lam, alt))) < 1e-14


def test_printed_table_does_not_map_back_stably():
    # the inverse embedding rescales the state by s_{i+1} = s_i^2 / a_i; with
    # the printed coefficients s leaves the FP64 range, which is why tables of
    # the one-term form are trained in that form
    from oracle import tables
    s = 1.0
    for a, _, _, _ in tables.PRINTED_B1500:
        s = s * s / a
    assert abs(s) < 1e-300


def test_golden_one_term_table():
    # written by tests/golden/make_alt_table.py (oracle only): trained in the
    # one-term form, its recorded max error is reproduced here
    with open(os.path.join(GOLDEN, "alt_table.json")) as f:
        d = json.load(f)
    alt = np.array(d["alt"])
    assert alt.shape == (d["L"] + 1, 2)
    err = altform.max_error(alt, "fermi", d["beta0"], d["mu0"], grid=200_001)
    assert abs(err - d["max_err"]) <= 1e-3 * d["max_err"] + 1e-15
    assert err < d["bound"]
    # the embedding gives the same function
    x = np.linspace(0.0, 1.0, 4001)
    assert np.max(np.abs(mlsp2.mlsp2_scalar(x, altform.to_mlsp2(alt)) - altform.alt_scalar(x, alt))) < 1e-12
    ent = np.array(d["alt_entropy"])
    e_err = altform.max_error(ent, "entropy", d["beta0"], d["mu0"], alpha=d["alpha"], grid=200_001)
    assert abs(e_err - d["max_err_entropy"]) <= 1e-3 * d["max_err_entropy"] + 1e-15


def test_library_conversion_matches_oracle():
    # ftsp2_alt_to_mlsp2 is host code: callable without a GPU
    ft = pytest.importorskip("paper_2605_08523_gb300")
    try:
        ft.lib()
    except Exception as e:            # library not built in this environment
        pytest.skip(str(e))
    rng = np.random.default_rng(11)
    for L in (1, 2, 9, 64):
        alt = rng.normal(size=(L + 1, 2))
        assert np.array_equal(ft.ftsp2_alt_to_mlsp2(alt), altform.to_mlsp2(alt))
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_alt_to_mlsp2(np.zeros((66, 2)))
    bad = np.zeros((3, 2))
    bad[1, 0] = np.nan
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_alt_to_mlsp2(bad)


def test_lm_fit_lowers_the_cost_from_the_sp2_start():
    # property of the LM loop (Marquardt acceptance): the accepted cost never
    # rises, and a few iterations from the exact SP2 sequence cut it by orders
    beta0, mu0, L = 40.0, 1.0 / 3.0, 8
    x = train.sample_grid(3000, beta0, mu0)
    a0 = altform.sp2_alt(mu0, L)
    a, hist = altform.lm_fit(a0, x, "fermi", beta0, mu0, iters=30, accel=True)
    costs = [h[0] for h in hist]
    assert all(b <= c for c, b in zip(costs, costs[1:]))
    c0 = 0.5 * np.sum((altform.forward(a0, x) - train.target(x, "fermi", beta0, mu0)) ** 2)
    assert costs[-1] < 1e-2 * c0
