"""GPU training of the families that keep stored layers (Sec. II A 2, II A 3,
II C) against the oracle: the Max-SP2 residuals on the GPU, Levenberg-Marquardt
steps of a Max-SP2 table (ftsp2_train_coeffs_max) and of a Skip-SP2 table with
two stored layers and two accumulators (ftsp2_train_coeffs_skipk) taken from
the library's own samples and starts, against the oracle's fits from its own,
and a full Max-SP2 fit reaching an error the Eq. mlsp2 table of the same
depth does not."""
import numpy as np
import pytest

from oracle import maxsp2, skipsp2, train

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.mark.parametrize("target", ["fermi", "entropy"])
def test_max_residuals_match_oracle(ft, target):
    rng = np.random.default_rng(3)
    L, beta0, mu0, alpha = 9, 100.0, 1 / 3, 0.842704
    p = maxsp2.mlsp2_to_max(train.init_from_sp2(L, beta0, mu0)) + 1e-3 * rng.standard_normal(maxsp2.nparams(L))
    x = np.linspace(0.0, 1.0, 30001)
    tcode = ft.TARGET_ENTROPY if target == "entropy" else ft.TARGET_FERMI
    r = ft.ftsp2_train_residuals(tcode, beta0, mu0, p, torch.from_numpy(x).cuda(), alpha=alpha, family=2)
    ref = maxsp2.forward(p, L, x, target, alpha, mu0) - train.target(x, target, beta0, mu0)
    assert np.max(np.abs(r.cpu().numpy() - ref)) < 1e-12


@pytest.mark.parametrize("seed", [0, 7])
def test_max_lm_steps_match_oracle(ft, seed):
    L, beta0, mu0, ns, it = 8, 100.0, 1 / 3, 4000, 3
    x = train.sample_grid(ns, beta0, mu0, seed=seed)
    p0 = maxsp2.mlsp2_to_max(train.init_from_sp2(L, beta0, mu0))
    p_or, hist = maxsp2.lm_fit(p0, L, x, "fermi", beta0, mu0, iters=it, accel=False)
    p_gpu, rep = ft.ftsp2_train_coeffs_max(ft.TARGET_FERMI, beta0, mu0, L=L, nsamples=ns, seed=seed, iterations=it,
                                           accel=False)
    assert rep["accepted"] == sum(int(h[2]) for h in hist)
    assert np.max(np.abs(p_gpu - p_or)) < 1e-8 * max(1.0, np.max(np.abs(p_or)))
    assert abs(rep["cost"] - hist[-1][0]) < 1e-9 * hist[-1][0]


def test_skipk_lm_steps_match_oracle(ft):
    L, k, K, beta0, mu0, ns, it = 8, 2, 2, 100.0, 1 / 3, 4000, 4
    x = train.sample_grid(ns, beta0, mu0)
    t0 = maxsp2.skip_from_skip1(skipsp2.from_mlsp2(train.init_from_sp2(L, beta0, mu0)), k, K, beta_extra=0.01)
    t_or, hist = maxsp2.skip_lm_fit(t0, "fermi", x, beta0, mu0, iters=it, accel=False)
    v_gpu, rep = ft.ftsp2_train_coeffs_skipk(ft.TARGET_FERMI, beta0, mu0, L, k, K, nsamples=ns, iterations=it,
                                             accel=False)
    q_or = maxsp2.skip_pack(t_or)
    assert rep["accepted"] == sum(int(h[2]) for h in hist)
    assert np.max(np.abs(v_gpu - q_or)) < 1e-7 * max(1.0, np.max(np.abs(q_or)))
    assert abs(rep["cost"] - hist[-1][0]) < 1e-8 * hist[-1][0]


def test_max_fit_beats_mlsp2_at_equal_depth(ft):
    # beta0 = 100, 10 layers: the GPU-fitted Max-SP2 table's max error on
    # [0, 1] is below the Eq. mlsp2 table's of the same depth
    L, beta0, mu0, ns = 10, 100.0, 1 / 3, 20000
    p, rep = ft.ftsp2_train_coeffs_max(ft.TARGET_FERMI, beta0, mu0, L=L, nsamples=ns, iterations=300, accel=True)
    th, rep_m = ft.ftsp2_train_coeffs(ft.TARGET_FERMI, beta0, mu0, L=L, nsamples=ns, iterations=300, accel=True)
    e_max = maxsp2.max_error(p, L, beta0=beta0, mu0=mu0, grid=200_001)
    e_ml = train.max_error(th, beta0=beta0, mu0=mu0, grid=200_001)
    assert e_max < 0.5 * e_ml, (e_max, e_ml)
    x = train.sample_grid(ns, beta0, mu0)
    assert abs(rep["max_err"] - np.max(np.abs(maxsp2.max_scalar(x, p, L) - train.fermi_target(x, beta0, mu0)))) < 1e-12
