"""Pins for the oracle's spectral bounds, rescaling, flip, validity, model choice
and the end-to-end Alg. 2 pipeline (CPU only)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import fermi, mlsp2, pipeline, rescale, sp2, tables

TH = tables.PRINTED_B1500
PRINTED = rescale.Table(TH, 1500.0, 1.0 / 3.0, name="printed")


def test_gershgorin_bruteforce_and_diagonal():
    rng = np.random.default_rng(1)
    M = rng.uniform(-2, 2, (4, 4))
    H = 0.5 * (M + M.T)
    assert np.allclose(rescale.gershgorin(H), rescale.gershgorin_loops(H.tolist()), rtol=0, atol=1e-15)
    d = rng.uniform(-3, 3, 9)
    assert rescale.gershgorin(np.diag(d)) == (d.min(), d.max())
    H = wl.lattice_3d((4, 4, 4), 0)
    lo, hi = rescale.gershgorin(H)
    w = np.linalg.eigvalsh(H)
    assert lo <= w[0] and w[-1] <= hi


def test_rescaling_identity():
    # Eq. rescaling: (H - mu I) beta = (mu' I - H') beta', and Eq. H0 gives
    # H0 = mu0 I + (beta/beta0)(mu I - H) (no flip) or (H - mu I) (flip).
    H = wl.chain_1d(40, 2)
    mu, kT = 0.3, 0.1
    beta = 1 / kT
    lo, hi = rescale.gershgorin(H)
    W = hi - lo
    I = np.eye(40)
    Hp = (hi * I - H) / W
    mup, betap = rescale.normalise(lo, hi, mu, beta)
    assert np.max(np.abs((H - mu * I) * beta - (mup * I - Hp) * betap)) < 1e-12
    for mu in (0.3, -0.4):
        H0, rec = rescale.rescale(H, mu, kT, [PRINTED])
        sign = -1.0 if rec.flip else 1.0
        assert np.max(np.abs(H0 - (I / 3.0 + sign * (beta / 1500.0) * (mu * I - H)))) < 1e-13
    assert rescale.rescale(H, 0.3, kT, [PRINTED])[1].flip != rescale.rescale(H, -0.4, kT, [PRINTED])[1].flip


def test_flip_identity():
    # Eq. flip: f(x'; beta', mu') = 1 - f(1 - x'; beta', 1 - mu').
    x = np.linspace(0, 1, 1001)
    for bp, mp in ((50.0, 0.7), (300.0, 0.55)):
        lhs = fermi.fermi(-x, -mp, 1 / bp)
        rhs = 1 - fermi.fermi(-(1 - x), -(1 - mp), 1 / bp)
        assert np.max(np.abs(lhs - rhs)) < 1e-15


def test_validity_matches_eq_conditions():
    rng = np.random.default_rng(4)
    for _ in range(2000):
        mup = rng.uniform(0.001, 0.999)
        bp = rng.uniform(1, 3000)
        eq = (1 / 3 / mup * 1500 >= bp) and ((2 / 3) / (1 - mup) * 1500 >= bp)
        assert rescale.is_valid(mup, bp, 1500.0, 1 / 3) == eq
    # beta' <= 2/3 beta0 is valid for every mu' in (0, 1/2] (Sec. IV C)
    for mup in np.linspace(0.01, 0.5, 50):
        assert rescale.is_valid(mup, 1000.0, 1500.0, 1 / 3)
    assert not rescale.is_valid(0.5, 1000.1, 1500.0, 1 / 3)


def test_model_choice_smallest_valid_beta0():
    t_small = rescale.Table(TH, 300.0, 1 / 3, name="small")
    t_big = rescale.Table(TH, 1500.0, 1 / 3, name="big")
    assert rescale.select_model([t_big, t_small], 0.4, 150.0) == 1
    assert rescale.select_model([t_big, t_small], 0.4, 800.0) == 0
    assert rescale.select_model([t_big, t_small], 0.4, 1400.0) == -1


def test_model_choice_fewest_layers_policy():
    # with the fewest-layers policy a longer low-beta0 table loses to a shorter
    # valid one; ties in the layer count go to the smaller beta0
    th26 = np.asarray(TH)
    th32 = np.vstack([th26, th26[:6]])
    t_low_long = rescale.Table(th32, 200.0, 1 / 3, name="b200_L32")
    t_mid = rescale.Table(th26, 1500.0, 1 / 3, name="b1500_L26")
    t_mid2 = rescale.Table(th26, 3000.0, 1 / 3, name="b3000_L26")
    ts = [t_low_long, t_mid2, t_mid]
    assert rescale.select_model(ts, 0.4, 100.0) == 0                    # default: smallest beta0
    assert rescale.select_model(ts, 0.4, 100.0, min_layers=True) == 2   # fewest layers, then beta0
    assert rescale.select_model(ts, 0.4, 1400.0, min_layers=True) == 1  # only b3000 is valid
    assert rescale.select_model(ts, 0.4, 9000.0, min_layers=True) == -1


def test_appendix_harness():
    # Appendix A test cases: 10 seeds, N = 100, beta ~ U(1, (2/3 beta0)/W),
    # mu ~ U(e_min, e_max); the 2-norm error against diagonalisation is at the
    # model error (< 2^-24).
    for seed in range(10):
        H = wl.appendix_matrix(seed)
        rng = wl.appendix_rng(seed)
        lo, hi = rescale.gershgorin(H)
        beta = rng.uniform(1, (2 / 3 * 1500) / (hi - lo))
        mu = rng.uniform(lo, hi)
        out = pipeline.density_entropy(H, mu, 1 / beta, [PRINTED], want_entropy=False)
        Dref, _, _, _ = fermi.eig_reference(H, mu, 1 / beta)
        assert np.linalg.norm(out["D"] - Dref, 2) < 1e-7


def test_density_invariants_lattice():
    H = wl.lattice_3d((4, 4, 4), 1)
    n = H.shape[0]
    kT = 0.1
    eps = np.linalg.eigvalsh(H)
    mu = fermi.mu_at_filling(eps, kT, n / 2)
    Dref, Sref, trref, _ = fermi.eig_reference(H, mu, kT)
    assert abs(np.trace(Dref) - np.sum(fermi.fermi(eps, mu, kT))) < 1e-10
    assert abs(trref - n / 2) < 1e-8
    assert np.max(np.abs(Dref @ H - H @ Dref)) < 1e-12
    out = pipeline.density_entropy(H, mu, kT, [PRINTED])
    ex = pipeline.method_exact(H, mu, kT, [PRINTED])
    assert np.max(np.abs(out["D"] - ex["D"])) < 1e-10        # rounding only
    assert np.max(np.abs(out["D"] - Dref)) < 5e-8            # model error
    assert np.max(np.abs(out["D"] @ H - H @ out["D"])) < 1e-8
    assert abs(out["S"] - ex["S"]) < 1e-8
    # S from theta_fermi + alpha ansatz: per-state error <= 1.24e-3
    assert abs(out["S"] - Sref) < 1.3e-3 * n


def test_zero_temperature_limit_idempotent():
    H = wl.chain_1d(60, 3)
    eps = np.linalg.eigvalsh(H)
    mu = 0.5 * (eps[29] + eps[30])
    errs = []
    for kT in (1e-2, 1e-3, 1e-4):
        D, _, _, _ = fermi.eig_reference(H, mu, kT)
        errs.append(np.max(np.abs(D @ D - D)))
    assert errs[-1] < 1e-12 and errs[0] > errs[-1]


def test_diagonal_H_reduces_to_scalar():
    d = np.linspace(-1.0, 1.0, 33)
    H = np.diag(d)
    mu, kT = 0.1, 0.05
    out = pipeline.density_entropy(H, mu, kT, [PRINTED])
    rec = out["rec"]
    x0 = rescale.x0_of_eigenvalue(d, mu, kT, rec, PRINTED)
    p = mlsp2.mlsp2_scalar(x0, TH)
    if rec.flip:
        p = 1 - p
    assert np.max(np.abs(np.diag(out["D"]) - p)) < 1e-12
    assert np.max(np.abs(np.diag(out["D"]) - fermi.fermi(d, mu, kT))) < 5e-8


def test_validity_region_error_printed_model(paper):
    # Fig. validity (bottom): inside the region of validity the (1500, 1/3)
    # model error stays below 10^-7.5.  Sampled on a (beta', mu') grid.
    x = np.linspace(0.0, 1.0, 20001)       # eigenvalues of H' in [0, 1]
    worst = 0.0
    for mup in np.linspace(0.02, 0.98, 25):
        for frac in (0.1, 0.5, 1.0):
            m = min(mup, 1 - mup)
            bp = frac * rescale.beta_max(m, 1500.0, 1 / 3)
            flip = mup > 0.5
            xp = 1 - x if flip else x
            mp = 1 - mup if flip else mup
            x0 = (bp / 1500.0) * (xp - mp) + 1 / 3
            p = mlsp2.mlsp2_scalar(x0, TH)
            if flip:
                p = 1 - p
            f = 1.0 / (1.0 + np.exp(-bp * (x - mup)))   # occupation in the H' frame
            worst = max(worst, np.max(np.abs(p - f)))
    assert worst < paper["validity_error_b1500"]


def test_invalid_and_clamped():
    H = wl.lattice_3d((4, 4, 4), 2)
    out = pipeline.density_entropy(H, 0.0, 0.001, [PRINTED], want_entropy=False)
    assert out["D"] is None and not out["rec"].valid
    out = pipeline.density_entropy(H, 0.0, 0.001, [PRINTED], clamp=True, want_entropy=False)
    rec = out["rec"]
    assert out["D"] is not None and not rec.valid
    assert abs(rec.beta_p - rescale.beta_max(rec.mu_p, 1500.0, 1 / 3)) < 1e-9


def test_degenerate_spectrum():
    H = 0.7 * np.eye(8)
    out = pipeline.density_entropy(H, 0.65, 0.1, [PRINTED])
    assert np.max(np.abs(out["D"] - fermi.fermi(0.7, 0.65, 0.1)[()] * np.eye(8))) < 5e-8


def test_mu_outside_spectrum():
    # mu above every Gershgorin bound: all states occupied, still valid when
    # the temperature is high enough (linear validity form).
    H = wl.chain_1d(20, 0)
    lo, hi = rescale.gershgorin(H)
    mu = hi + 0.2
    out = pipeline.density_entropy(H, mu, 0.5, [PRINTED], want_entropy=False)
    Dref, _, _, _ = fermi.eig_reference(H, mu, 0.5)
    assert out["rec"].valid and out["rec"].mu_p < 0
    assert np.max(np.abs(out["D"] - Dref)) < 5e-8


def test_sp2_mu_sequence_keeps_mu_fixed_and_forms_step():
    # Eq. sp2-mu keeps the image of mu' near mu' (so mu' becomes the location
    # of the step); points above mu' go to 1, below to 0.
    for mup in (0.2, 1 / 3, 0.6):
        sig, m = sp2.sp2_mu_sequence(mup, 40)
        assert abs(m - mup) < 0.35
        th = sp2.sp2_table(mup, 40)
        x = np.array([mup - 0.05, mup + 0.05])
        p = mlsp2.mlsp2_scalar(x, th)
        assert p[0] < 1e-6 and p[1] > 1 - 1e-6
    # the embedding reproduces X^2 / 2X - X^2 exactly on matrices
    rng = np.random.default_rng(2)
    M = rng.standard_normal((6, 6))
    X = np.eye(6) * 0.4 + 0.02 * (M + M.T)
    th = sp2.sp2_table(0.4, 3)
    sig, _ = sp2.sp2_mu_sequence(0.4, 3)
    Y = X.copy()
    for s in sig:
        Y = Y @ Y if s > 0 else 2 * Y - Y @ Y
    assert np.max(np.abs(mlsp2.mlsp2_matrix(X, th) - Y)) < 1e-14
