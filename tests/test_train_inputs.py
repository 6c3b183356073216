"""The training inputs the library builds on the host (no GPU needed), against
the oracle: the sample set of Sec. II C 1 (ftsp2_train_samples against
oracle.train.sample_grid, seed 0 and seeded), the starting tables
(ftsp2_train_init against oracle.train.init_from_sp2, ftsp2_train_init_alt
against oracle.altform.sp2_alt) and the Appendix embedding
(ftsp2_mlsp2_to_skip against oracle.skipsp2.from_mlsp2).  These are the
inputs of every table the library trains when the caller passes no start."""
import numpy as np
import pytest

from oracle import altform, skipsp2, sp2, tables, train


@pytest.fixture(scope="module")
def ft():
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.mark.parametrize("beta0,mu0,N,seed", [(200.0, 1 / 3, 100_000, 0), (1500.0, 1 / 3, 4000, 0),
                                              (20.0, 0.5, 777, 0), (100.0, 1 / 3, 5000, 99)])
def test_samples_match_oracle(ft, beta0, mu0, N, seed):
    x = ft.ftsp2_train_samples(beta0, mu0, N, seed)
    xo = train.sample_grid(N, beta0, mu0, seed=seed)
    assert np.max(np.abs(x - xo)) <= 1e-15
    assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("L,beta0", [(12, 40.0), (16, 200.0), (26, 1500.0), (34, 3000.0), (44, 24000.0), (5, 20.0)])
def test_init_matches_oracle(ft, L, beta0):
    th = ft.ftsp2_train_init(L, beta0, 1 / 3)
    assert np.max(np.abs(th - train.init_from_sp2(L, beta0, 1 / 3))) <= 1e-15


@pytest.mark.parametrize("L,mu0", [(16, 1 / 3), (26, 1 / 3), (9, 0.6)])
def test_init_alt_matches_oracle(ft, L, mu0):
    assert np.array_equal(ft.ftsp2_train_init_alt(L, mu0), altform.sp2_alt(mu0, L))


@pytest.mark.parametrize("which", ["printed", "sp2"])
def test_skip_embedding_matches_oracle(ft, which):
    th = np.array(tables.PRINTED_B1500) if which == "printed" else train.init_from_sp2(16, 100.0, 1 / 3)
    got = ft.ftsp2_mlsp2_to_skip(th)
    assert np.max(np.abs(got - skipsp2.from_mlsp2(th))) <= 1e-15 * max(1.0, np.max(np.abs(got)))


def test_layer_count_matches_oracle(ft):
    for bp in (20.0, 308.3, 1500.0, 24000.0):
        assert abs(ft.ftsp2_layer_count(bp) - sp2.layer_count(bp)) <= 1e-13


def test_argument_checks(ft):
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_train_samples(-1.0, 1 / 3, 10)
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_train_init(0, 100.0, 1 / 3)
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_train_init(65, 100.0, 1 / 3)
    with pytest.raises(ft.Ftsp2Error):
        ft.ftsp2_mlsp2_to_skip(np.array([[0.0, 1.0, 0.0, 0.0]]))      # a linear layer has no square form


@pytest.mark.parametrize("L", [1, 5, 20])
def test_mlsp2_to_max_matches_oracle(ft, L):
    from oracle import maxsp2
    rng = np.random.default_rng(L)
    th = rng.normal(size=(L, 4)) * 0.5
    th[:, 0] = np.where(np.abs(th[:, 0]) < 0.2, 0.7, th[:, 0])
    got = ft.ftsp2_mlsp2_to_max(th)
    assert got.size == ft.max_nparams(L)
    assert np.max(np.abs(got - maxsp2.mlsp2_to_max(th))) <= 1e-13 * max(1.0, np.max(np.abs(got)))


@pytest.mark.parametrize("L,k,K", [(1, 1, 1), (6, 2, 2), (9, 3, 1), (4, 1, 3), (7, 2, 0), (20, 2, 2)])
def test_skip_to_max_matches_oracle(ft, L, k, K):
    from oracle import maxsp2
    rng = np.random.default_rng(100 * L + 10 * k + K)
    t = dict(alpha=rng.normal(size=(L, k + 1)), beta=rng.normal(size=(L, K)), gamma=rng.normal(size=(L, K)),
             A0=rng.normal(size=K), gL=float(rng.normal()))
    got = ft.ftsp2_skip_to_max(t["alpha"], t["beta"], t["gamma"], t["A0"], t["gL"])
    assert np.max(np.abs(got - maxsp2.skip_to_max(t))) <= 1e-13 * max(1.0, np.max(np.abs(got)))


def test_max_conversions_reject_bad_arguments(ft):
    with pytest.raises(Exception):
        ft.ftsp2_mlsp2_to_max(np.ones((21, 4)))          # more than 20 layers
    with pytest.raises(Exception):
        ft.ftsp2_skip_to_max(np.ones((3, 1)), np.ones((3, 1)), np.ones((3, 1)), np.ones(1))   # k = 0
    with pytest.raises(Exception):
        ft.ftsp2_skip_to_max(np.full((3, 2), np.nan), np.ones((3, 1)), np.ones((3, 1)), np.ones(1))
    assert [ft.max_layers_of(ft.max_nparams(L)) for L in (1, 7, 20)] == [1, 7, 20]


@pytest.mark.parametrize("L,k,K,beta0", [(12, 2, 2, 100.0), (8, 1, 1, 40.0), (10, 3, 2, 200.0)])
def test_skipk_start_and_embedding_match_oracle(ft, L, k, K, beta0):
    from oracle import maxsp2
    v = ft.ftsp2_train_init_skipk(L, k, K, beta0, 1 / 3)
    t = maxsp2.skip_from_skip1(skipsp2.from_mlsp2(train.init_from_sp2(L, beta0, 1 / 3)), k, K, beta_extra=0.01)
    assert v.size == (1 + k + 2 * K) * L + 2
    assert np.max(np.abs(v - maxsp2.skip_pack(t))) <= 1e-14 * max(1.0, np.max(np.abs(v)))
    # the start computes the Eq. mlsp2 start's function
    p = ft.ftsp2_skipk_to_max(v, L, k, K)
    assert np.max(np.abs(p - maxsp2.skip_to_max(t))) <= 1e-13 * max(1.0, np.max(np.abs(p)))
    x = np.linspace(0.0, 1.0, 1001)
    ref = train.forward(train.init_from_sp2(L, beta0, 1 / 3), x)
    assert np.max(np.abs(maxsp2.max_scalar(x, p, L) - ref)) < 1e-11


def test_skipk_entry_points_reject_bad_shapes(ft):
    with pytest.raises(Exception):
        ft.ftsp2_train_init_skipk(3, 4, 2, 100.0, 1 / 3)          # more stored layers than layers
    with pytest.raises(Exception):
        ft.ftsp2_train_init_skipk(5, 2, 0, 100.0, 1 / 3)          # no accumulator
    with pytest.raises(Exception):
        ft.ftsp2_train_init_skipk(21, 2, 2, 100.0, 1 / 3)         # beyond the 20-layer limit
    with pytest.raises(ValueError):
        ft.ftsp2_skipk_to_max(np.zeros(10), 5, 2, 2)              # wrong vector length
    v = ft.ftsp2_train_init_skipk(5, 2, 2, 100.0, 1 / 3)
    assert v.size == ft.skipk_nparams(5, 2, 2) == (1 + 2 + 4) * 5 + 2
