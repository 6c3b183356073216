"""Pins for the oracle's training pieces (CPU only): sampling density, reverse-
mode Jacobian against finite differences, and Levenberg-Marquardt on problems
with a known exact fit."""
import math

import numpy as np
import pytest

from oracle import mlsp2, sp2, tables, train

TH = np.array(tables.PRINTED_B1500)


def test_sample_grid_density():
    # Quantile grid of p ~ 1 + |f'|: the fraction of samples in an interval is
    # the integral of p over it.
    N = 100000
    x = train.sample_grid(N, 200.0, 1 / 3)
    assert np.all(np.diff(x) > 0) and 0 < x[0] and x[-1] < 1
    Z = 1.0 + (1 / (1 + math.exp(-200 * (2 / 3))) - 1 / (1 + math.exp(200 / 3)))
    a, b = 0.3, 0.4
    mass = (b - a) + (1 / (1 + math.exp(-200 * (b - 1 / 3))) - 1 / (1 + math.exp(-200 * (a - 1 / 3))))
    frac = np.mean((x >= a) & (x < b))
    assert abs(frac - mass / Z) < 2e-4
    u = train.sample_grid(1000, 200.0, 1 / 3, weighting="uniform")
    assert np.max(np.abs(u - (np.arange(1000) + 0.5) / 1000)) < 1e-6


def test_fermi_target_matches_printed_model():
    x = np.linspace(0, 1, 200001)
    assert np.max(np.abs(train.forward(TH, x) - train.fermi_target(x, 1500.0, 1 / 3))) < 3e-8
    assert abs(train.max_error(TH, grid=400001) - 2.23e-8) < 0.05e-8


@pytest.mark.parametrize("kind", ["fermi", "entropy"])
def test_jacobian_vs_central_differences(kind):
    rng = np.random.default_rng(0)
    L = 6
    th = np.array(sp2.sp2_table(1 / 3, L)) + 0.05 * rng.standard_normal((L, 4))
    x = rng.uniform(0, 1, 64)
    y, J = train.forward_jacobian(th, x, kind, alpha=0.84, mu0=1 / 3)
    assert np.max(np.abs(y - train.forward(th, x, kind, 0.84, 1 / 3))) < 1e-14
    h = 1e-6
    flat = th.ravel()
    for j in range(4 * L):
        e = np.zeros_like(flat)
        e[j] = h
        fd = (train.forward((flat + e).reshape(L, 4), x, kind, 0.84, 1 / 3)
              - train.forward((flat - e).reshape(L, 4), x, kind, 0.84, 1 / 3)) / (2 * h)
        assert np.max(np.abs(fd - J[:, j])) < 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_jacobian_single_layer_closed_form():
    # One layer: F = d x + a x^2 + b x + c, so dF/dtheta = (x^2, x, 1, x).
    th = np.array([[0.7, -0.3, 0.2, 0.5]])
    x = np.linspace(0, 1, 11)
    _, J = train.forward_jacobian(th, x)
    assert np.max(np.abs(J - np.stack([x * x, x, np.ones_like(x), x], 1))) == 0.0


@pytest.mark.parametrize("accel", [False, True])
def test_lm_recovers_teacher(accel):
    # Targets produced by a known table: LM from a perturbed start must drive
    # the residual to rounding level (an exact fit exists).
    rng = np.random.default_rng(1)
    L = 5
    teacher = np.array(sp2.sp2_table(0.4, L)) + 0.02 * rng.standard_normal((L, 4))
    x = np.linspace(0, 1, 400)
    y = train.forward(teacher, x)
    start = teacher + 0.01 * rng.standard_normal((L, 4))

    class T:
        pass
    orig = train.target
    try:
        train.target = lambda xx, kind, b0, m0: train.forward(teacher, xx)
        th, hist = train.lm_fit(start, x, iters=60, accel=accel)
    finally:
        train.target = orig
    assert np.max(np.abs(train.forward(th, x) - y)) < 1e-9
    assert hist[-1][0] < 1e-20


def test_lm_single_step_linear_problem():
    # With only linear parameters varied (c_i, d_i enter linearly when every
    # a_i = 0), one LM step with lambda -> 0 lands on the least-squares optimum.
    rng = np.random.default_rng(3)
    L = 3
    th = np.zeros((L, 4))
    th[:, 1] = [0.9, 1.1, 0.8]
    x = np.linspace(0, 1, 50)
    y, J = train.forward_jacobian(th, x)
    tgt = rng.standard_normal(50)
    keep = [2, 3, 6, 7, 10, 11]
    Jk = J[:, keep]
    JTJ, g = train.normal_equations(Jk, y - tgt)
    v = train.lm_direction(JTJ + 1e-14 * np.eye(len(keep)), g, 0.0)
    sol, *_ = np.linalg.lstsq(Jk, tgt - y, rcond=None)
    assert np.max(np.abs(Jk @ v - Jk @ sol)) < 1e-9


def test_training_improves_on_sp2_beta40():
    # What training gains (Fig. 2 in spirit): at beta0 = 40, mu0 = 1/3 with 12
    # layers, the untrained SP2-mu sequence misses the Fermi function by ~1e-1;
    # a few LM iterations from a slope-matched start bring it below 1e-4.
    L = 12
    beta0, mu0 = 40.0, 1 / 3
    x = train.sample_grid(4000, beta0, mu0)
    start = np.array(sp2.sp2_table(mu0, L))
    e0 = train.max_error(start, beta0=beta0, mu0=mu0, grid=20001)
    th, hist = train.lm_fit(train.init_from_sp2(L, beta0, mu0), x, beta0=beta0, mu0=mu0,
                            iters=150, accel=True)
    e1 = train.max_error(th, beta0=beta0, mu0=mu0, grid=20001)
    assert e0 > 5e-2 and e1 < 1e-4


def _cdf_closed_form(x, beta0, mu0):
    # F(x) for p ~ 1 + f' (f the increasing logistic, f' > 0): integral of p
    # from 0 to x over its value at 1
    f = lambda t: 1.0 / (1.0 + np.exp(-beta0 * (t - mu0)))
    return (x + f(x) - f(0.0)) / (1.0 + f(1.0) - f(0.0))


@pytest.mark.parametrize("seed", [0, 7, 12345])
def test_sample_grid_points_in_their_quantile_cells(seed):
    # Point s lies in the s-th of N equal-probability cells of p (closed-form
    # CDF); seed 0 puts it at the cell's middle, a seed draws its position.
    N, beta0, mu0 = 2000, 200.0, 1 / 3
    x = train.sample_grid(N, beta0, mu0, seed=seed)
    q = _cdf_closed_form(x, beta0, mu0) * N - np.arange(N)
    assert np.all(q > -1e-6) and np.all(q < 1 + 1e-6)
    if seed == 0:
        assert np.max(np.abs(q - 0.5)) < 1e-4
    else:
        assert np.std(q) > 0.2          # positions spread over the cells
        assert np.array_equal(x, train.sample_grid(N, beta0, mu0, seed=seed))


def test_seeded_grid_uses_splitmix64():
    # the cell offsets are the generator's published outputs (first value of
    # splitmix64 for state 1: 0x910a2dec89025cc1)
    from oracle import lanczos
    assert lanczos.splitmix64(1) == 0x910A2DEC89025CC1
    x = train.sample_grid(4, 50.0, 0.4, weighting="uniform", seed=1)
    u0 = (lanczos.splitmix64(1) >> 11) * 2.0 ** -53
    assert abs(x[0] - u0 / 4) < 1e-6


@pytest.mark.parametrize("L,beta0", [(12, 40.0), (24, 200.0), (30, 3000.0)])
def test_sp2_init_slope_is_beta0_over_4(L, beta0):
    # the contraction folded into layer 0 makes the slope at mu0 equal to the
    # target's beta0 / 4 whenever the SP2 sequence alone is steeper (central
    # differences of the composed polynomial, independent of the chain rule)
    mu0 = 1 / 3
    th = train.init_from_sp2(L, beta0, mu0)
    s_sp2 = sp2.slope_at(np.array(sp2.sp2_table(mu0, L)), mu0, h=1e-9)
    s = sp2.slope_at(th, mu0, h=1e-9)
    if s_sp2 > beta0 / 4:
        assert abs(s - beta0 / 4) < 1e-5 * beta0
    else:
        assert np.array_equal(th, np.array(sp2.sp2_table(mu0, L)))
    # mu0 stays a point of the SP2 trajectory: the same image as without contraction
    assert abs(mlsp2.mlsp2_scalar([mu0], th)[0] - mlsp2.mlsp2_scalar([mu0], sp2.sp2_table(mu0, L))[0]) < 1e-12
