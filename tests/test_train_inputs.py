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
