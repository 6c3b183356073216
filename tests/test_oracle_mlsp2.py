"""Pins for the oracle's scalar/matrix MLSP2 recursion, the entropy model and the
layer-count formulas, against values the paper prints, closed forms and brute
force (CPU only)."""
import math

import numpy as np
import pytest

from oracle import fermi, mlsp2, sp2, tables


TH = tables.PRINTED_B1500


def logistic(x, beta0, mu0):
    return 1.0 / (1.0 + np.exp(-beta0 * (x - mu0)))


def test_printed_table_shape():
    assert len(TH) == 26 and all(len(r) == 4 for r in TH)


def test_printed_weights_fit_increasing_logistic(paper):
    # Sec. IV D: with 26 layers the model error is below 2^-24.  Pins the
    # variable convention (no inner flip) and the layer order of Eq. mlsp2.
    x = np.linspace(0.0, 1.0, 2_000_001)
    err = np.max(np.abs(mlsp2.mlsp2_scalar(x, TH) - logistic(x, paper["printed_model_beta0"],
                                                               paper["printed_model_mu0"])))
    assert err < paper["printed_model_error_bound"]
    assert 1e-8 < err < 3e-8            # 2.23e-8 measured


@pytest.mark.parametrize("variant", ["inner_flip", "decreasing", "mirror_mu",
                                     "acc_after_update", "drop_c", "swap_ab"])
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_plausible_mistakes_are_caught(variant):
    # Each plausible misreading of Eq. mlsp2 / Alg. 1 misses the target by O(1).
    x = np.linspace(0.0, 1.0, 20001)
    tgt = logistic(x, 1500.0, 1.0 / 3.0)
    if variant == "inner_flip":
        y = mlsp2.mlsp2_scalar(1.0 - x, TH)
    elif variant == "decreasing":
        y = 1.0 - mlsp2.mlsp2_scalar(x, TH)
    elif variant == "mirror_mu":
        y = mlsp2.mlsp2_scalar(x, TH)
        tgt = logistic(x, 1500.0, 2.0 / 3.0)
    else:
        xi = x.copy()
        A = np.zeros_like(x)
        for a, b, c, d in TH:
            if variant == "acc_after_update":
                xi = a * xi * xi + b * xi + c
                A = A + d * xi
            elif variant == "drop_c":
                A = A + d * xi
                xi = a * xi * xi + b * xi
            elif variant == "swap_ab":
                A = A + d * xi
                xi = b * xi * xi + a * xi + c
        y = A + xi
    with np.errstate(invalid="ignore"):
        err = np.abs(y - tgt)
    assert (not np.all(np.isfinite(err))) or err.max() > 1e-3


def test_scalar_fp32_floor():
    # The same recursion in FP32 from FP32 inputs: ~2.7e-5 worst case, largest
    # near mu0 where the slope beta0/4 amplifies rounding.
    x = np.linspace(0.0, 1.0, 200001)
    d = np.abs(mlsp2.mlsp2_scalar(x, TH, dtype=np.float32) - mlsp2.mlsp2_scalar(x, TH))
    assert 5e-6 < d.max() < 1e-4
    assert abs(x[np.argmax(d)] - 1.0 / 3.0) < 0.05


def test_matrix_recursion_on_diagonal_is_scalar():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 37)
    F = mlsp2.mlsp2_matrix(np.diag(x), TH)
    assert np.max(np.abs(np.diag(F) - mlsp2.mlsp2_scalar(x, TH))) < 1e-12
    assert np.max(np.abs(F - np.diag(np.diag(F)))) == 0.0


def _matmul_loops(A, B):
    n = len(A)
    return [[sum(A[i][k] * B[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def test_matrix_recursion_bruteforce_4x4():
    # Explicit triple-loop products and a pure-Python Jacobi eigensolver,
    # independent of BLAS/LAPACK.
    rng = np.random.default_rng(11)
    M = rng.uniform(-1, 1, (4, 4))
    H = 0.5 * (M + M.T)
    w, V = fermi.jacobi_eigh(H.tolist())
    w = np.array(w)
    # map the spectrum into (0.25, 0.45), where the model is steep
    X0 = 0.25 + 0.2 * (H - w.min() * np.eye(4)) / (w.max() - w.min())
    X = X0.tolist()
    A = [[0.0] * 4 for _ in range(4)]
    for a, b, c, d in TH:
        A = [[A[i][j] + d * X[i][j] for j in range(4)] for i in range(4)]
        XX = _matmul_loops(X, X)
        X = [[a * XX[i][j] + b * X[i][j] + (c if i == j else 0.0) for j in range(4)] for i in range(4)]
    F_loops = np.array(A) + np.array(X)
    F = mlsp2.mlsp2_matrix(X0, TH)
    assert np.max(np.abs(F - F_loops)) < 1e-9
    # eigen route: V diag(P(x)) V^T with the Jacobi eigenvectors of X0
    wx, Vx = fermi.jacobi_eigh(X0.tolist())
    Vx = np.array(Vx)
    F_eig = (Vx * mlsp2.mlsp2_scalar(np.array(wx), TH)[None, :]) @ Vx.T
    assert np.max(np.abs(F - F_eig)) < 1e-9


def test_equivariance_and_commutation():
    # f(Q H Q^T) = Q f(H) Q^T (Appendix B) and [F(X), X] = 0.
    rng = np.random.default_rng(5)
    n = 24
    M = rng.standard_normal((n, n))
    X0 = np.eye(n) / 3.0 + 0.05 * (M + M.T) / math.sqrt(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    F = mlsp2.mlsp2_matrix(X0, TH)
    FQ = mlsp2.mlsp2_matrix(Q @ X0 @ Q.T, TH)
    assert np.max(np.abs(FQ - Q @ F @ Q.T)) < 1e-9
    assert np.max(np.abs(F @ X0 - X0 @ F)) < 1e-10


def test_entropy_function_properties():
    assert abs(fermi.entropy_of_t(0.0) - math.log(2.0)) < 1e-15   # s(mu) = ln 2
    t = np.linspace(-40, 40, 8001)
    assert np.max(np.abs(fermi.entropy_of_t(t) - fermi.entropy_of_t(-t))) == 0.0
    f = 1.0 / (np.exp(t) + 1.0)
    m = (f > 1e-300) & (f < 1 - 1e-16)
    assert np.max(np.abs(fermi.entropy_of_t(t[m]) - fermi.entropy_of_f(f[m]))) < 1e-12


def test_entropy_ansatz_alpha_values(paper):
    # Sec. II B and Table entropy: alpha = 1/sqrt(2 ln2) matches s''(mu);
    # alpha = 0.842704 minimises the max error, which is 1.24e-3.
    assert abs(mlsp2.ALPHA_CURVATURE - paper["alpha_curvature"]) < 1e-6
    t = np.linspace(-60, 60, 1_200_001)
    s = fermi.entropy_of_t(t)

    def maxerr(al):
        return np.max(np.abs(mlsp2.ansatz_entropy_of_t(t, al) - s))

    e_mm = maxerr(paper["alpha_minmax"])
    assert abs(e_mm - paper["entropy_theta_fermi_max_err"]) < 5e-6
    assert maxerr(mlsp2.ALPHA_CURVATURE) > 3 * e_mm
    # curvature at t = 0 matches for the curvature alpha
    h = 1e-3
    c_s = (fermi.entropy_of_t(h) - 2 * fermi.entropy_of_t(0.0) + fermi.entropy_of_t(-h)) / h**2
    c_a = (mlsp2.ansatz_entropy_of_t(h, mlsp2.ALPHA_CURVATURE)
           - 2 * mlsp2.ansatz_entropy_of_t(0.0, mlsp2.ALPHA_CURVATURE)
           + mlsp2.ansatz_entropy_of_t(-h, mlsp2.ALPHA_CURVATURE)) / h**2
    assert abs(c_s - c_a) < 1e-5
    # 0.842704 is the minimax point: neighbours are worse
    assert maxerr(0.8420) > e_mm and maxerr(0.8434) > e_mm


def test_entropy_m1_polynomial(paper):
    # Table entropy row 1: 4 ln2 f (1 - f) vs s(f): max err 7.55e-2; relative
    # error of S on 2048 evenly spaced eigenvalues at beta=40, mu=1/3: 0.157.
    f = np.linspace(0.0, 1.0, 2_000_001)
    e = np.max(np.abs(4 * math.log(2) * f * (1 - f) - fermi.entropy_of_f(f)))
    assert abs(e - paper["entropy_m1_max_err"]) < 1e-4
    x = np.linspace(0.0, 1.0, paper["entropy_table_npoints"])
    beta, mu = paper["entropy_table_beta"], paper["entropy_table_mu"]
    ff = fermi.fermi(x, mu, 1.0 / beta)
    S = np.sum(fermi.entropy(x, mu, 1.0 / beta))
    S1 = np.sum(4 * math.log(2) * ff * (1 - ff))
    assert abs(abs(S - S1) / S - paper["entropy_m1_rel_err"]) < 5e-4


def test_entropy_recursion_with_exact_fermi_stage():
    # The entropy recursion is Eq. entropy expansion: with a table that
    # reproduces the Fermi function, s~ = 4ln2 F(1-F) at y = alpha(x-mu0)+mu0
    # equals the ansatz.  The printed table stands in for "exact" up to 2.3e-8.
    x = np.linspace(0.0, 1.0, 100001)
    al = 0.842704
    s_rec = mlsp2.entropy_scalar(x, TH, al, 1.0 / 3.0)
    s_ans = mlsp2.ansatz_entropy_of_t(1500.0 * (x - 1.0 / 3.0), al)
    assert np.max(np.abs(s_rec - s_ans)) < 1e-7


def test_entropy_matrix_trace_identity():
    # S = 4ln2 (Tr F - Tr F^2) equals the sum of s~ over eigenvalues.
    rng = np.random.default_rng(8)
    n = 30
    M = rng.standard_normal((n, n))
    X0 = np.eye(n) / 3.0 + 0.04 * (M + M.T) / math.sqrt(n)
    S = mlsp2.entropy_matrix(X0, TH, 0.842704, 1.0 / 3.0)
    w = np.linalg.eigvalsh(X0)
    assert abs(S - np.sum(mlsp2.entropy_scalar(w, TH, 0.842704, 1.0 / 3.0))) < 1e-9
    assert S > 0


def test_layer_count(paper):
    # Eq. layer count and its printed uses.
    assert math.ceil(sp2.layer_count(40.0)) == paper["layers_needed_beta40"]
    assert math.ceil(sp2.layer_count(1500.0)) == paper["layers_needed_beta1500"]
    c1 = 1.0 / math.log(2 * sp2.PHI)
    c0 = -math.log(4.0) / math.log(2 * sp2.PHI)
    assert abs(c1 - paper["layer_count_slope"]) < 0.05
    assert abs(c0 - paper["layer_count_offset"]) < 0.05
    assert abs(sp2.beta0_for_layers(10) - paper["ten_layer_beta0"]) < 0.05
    assert abs(2 / 3 * sp2.beta0_for_layers(10) - paper["ten_layer_beta_prime"]) < 0.05


def test_golden_ratio_fixed_point():
    # Sec. IV B: (f1 o f0)(phi) = phi, f0'(phi) = f1'(phi^2) = 2 phi, and the
    # alternating composition has slope (2 phi)^n at phi.
    p = sp2.PHI
    assert abs(sp2.f1(sp2.f0(p)) - p) < 1e-15
    assert abs(2 * p - 2 * (1 - p * p)) < 1e-15
    for n in (2, 6, 10):
        h = 1e-7
        sl = (sp2.alternating_composition(p + h, n) - sp2.alternating_composition(p - h, n)) / (2 * h)
        assert abs(sl / (2 * p) ** n - 1) < 1e-5


def test_quadratic_convergence_to_step():
    # Appendix: repeated f1 o f0 drives x < phi to 0 and x > phi to 1, and
    # |F(x)| = 2 x^2 + O(x^3) near 0.
    x = np.array([0.2, 0.5, 0.7, 0.9])
    y = x.copy()
    for _ in range(12):
        y = sp2.f1(sp2.f0(y))
    assert np.all(y[x < sp2.PHI] < 1e-12) and np.all(y[x > sp2.PHI] > 1 - 1e-12)
    for e in (1e-3, 1e-4):
        assert abs(sp2.f1(sp2.f0(e)) / (2 * e * e) - 1) < 1e-2


def test_temperature_limit(paper):
    kB = 8.617e-5
    assert abs(1.0 / (kB * 1000.0) - paper["temperature_limit_K_per_eV"]) < 0.05
    assert abs(2 / 3 * paper["printed_model_beta0"] - paper["printed_model_beta_prime_limit"]) < 1e-9
