"""GPU parity of Skip-SP2 tables (one stored layer, one accumulator;
FTSP2_FAMILY_SKIP) against the oracle's Skip-SP2 recursion on the eigenvalues;
the embedded printed table against the Eq. mlsp2 path; a batch mixing both
families; and the library's Skip-SP2 training against the oracle's LM."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import fermi, pipeline, rescale, skipsp2, tables, train

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(ROOT, "tests", "golden", "skip_table.json")) as f:
        return json.load(f)


def skip_set(ft, d):
    return ft.ModelSet([dict(skip=d["skip"], skip_entropy=d["skip_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                             alpha=d["alpha"])])


def run(ft, ms, Hs, mus, kTs, mode, flags):
    flat, _ = wl.pack_batch(Hs)
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=3, flags=flags)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("shape", ["pair", "single"])
def test_skip_tables_match_oracle(ft, golden, mode, shape):
    if mode == "fp32" and shape == "single":
        pytest.skip("one shape on the CUDA cores")
    d = golden
    Hs = [wl.chain_1d(300, 4), wl.lattice_3d((8, 8, 8), 2)]
    mus, kTs = [0.1, -0.2], [0.2, 0.3]
    s = run(ft, skip_set(ft, d), Hs, mus, kTs, mode, ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES)
    for b, H in enumerate(Hs):
        ex = skipsp2.method_exact(H, mus[b], kTs[b], d["skip"], d["beta0"], d["mu0"], d["alpha"], d["skip_entropy"])
        assert ex["D"] is not None
        assert s.records()[b]["status"] == 0
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - D.T)) == 0.0
        assert np.max(np.abs(D - ex["D"])) < 1e-6, (mode, shape, b)
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6
        Dref, _, _, _ = fermi.eig_reference(H, mus[b], kTs[b])
        assert np.max(np.abs(D - Dref)) < d["max_err"] + 1e-6


@pytest.mark.parametrize("flags", ["deferred", "refine_tc"])
def test_skip_tables_deferred_and_refined(ft, golden, flags):
    d = golden
    H = wl.lattice_3d((8, 8, 16), 1)
    mu, kT = 0.05, 0.45
    f = ft.PAIR_TILES | (ft.EPI_DEFERRED if flags == "deferred" else ft.REFINE2 | ft.REFINE_TC)
    s = run(ft, skip_set(ft, d), [H], [mu], [kT], "fp16x2", f)
    ex = skipsp2.method_exact(H, mu, kT, d["skip"], d["beta0"], d["mu0"], d["alpha"], d["skip_entropy"])
    assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - ex["D"])) < 1e-6
    assert abs(float(s.S.cpu()[0]) - ex["S"]) / H.shape[0] < 1e-6


def test_embedded_printed_table(ft):
    # the printed table in Skip-SP2 form (Appendix embedding, beta = 0) and in
    # Eq. mlsp2 form: both match the oracle's Eq. mlsp2 method-exact result
    th = np.array(tables.PRINTED_B1500)
    emb = skipsp2.from_mlsp2(th)
    H = wl.lattice_3d((8, 8, 8), 6)
    mu, kT = 0.0, 0.1
    ex = pipeline.method_exact(H, mu, kT, [PRINTED])
    for tab in (dict(theta=th), dict(skip=emb)):
        ms = ft.ModelSet([dict(tab, beta0=1500.0, mu0=1.0 / 3.0, alpha=0.842704)])
        for mode in ("fp16x2", "bf16x3"):
            s = run(ft, ms, [H], [mu], [kT], mode, ft.PAIR_TILES)
            assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - ex["D"])) < 1e-6, (list(tab), mode)
            assert abs(float(s.S.cpu()[0]) - ex["S"]) / 512 < 1e-6


@pytest.mark.parametrize("shape", ["pair", "single"])
def test_batch_mixing_families(ft, golden, shape):
    # one launch per layer serves an instance on the Skip-SP2 table (small
    # beta') and one on the printed Eq. mlsp2 table (beta' beyond the Skip
    # table's region)
    d = golden
    ms = ft.ModelSet([dict(theta=tables.PRINTED_B1500, beta0=1500.0, mu0=1.0 / 3.0, alpha=0.842704),
                      dict(skip=d["skip"], skip_entropy=d["skip_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                           alpha=d["alpha"])])
    Hs = [wl.chain_1d(300, 4), wl.lattice_3d((8, 8, 8), 2)]
    mus, kTs = [0.1, -0.2], [0.2, 0.08]
    s = run(ft, ms, Hs, mus, kTs, "fp16x2", ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES)
    rec = s.records()
    assert list(rec["model"]) == [1, 0]
    ex0 = skipsp2.method_exact(Hs[0], mus[0], kTs[0], d["skip"], d["beta0"], d["mu0"], d["alpha"], d["skip_entropy"])
    ex1 = pipeline.method_exact(Hs[1], mus[1], kTs[1], [PRINTED])
    for b, ex in enumerate((ex0, ex1)):
        assert np.max(np.abs(s.matrix(b).double().cpu().numpy() - ex["D"])) < 1e-6, b
    assert abs(float(s.S.cpu()[0]) - ex0["S"]) / 300 < 1e-6


def test_skip_training_matches_oracle(ft):
    beta0, mu0, L = 60.0, 1.0 / 3.0, 10
    x = train.sample_grid(4000, beta0, mu0)
    t0 = skipsp2.from_mlsp2(train.init_from_sp2(L, beta0, mu0))
    ref, hist = skipsp2.lm_fit(t0, x, "fermi", beta0, mu0, iters=8, accel=False)
    # no start table: the library embeds its own SP2 start (= the oracle's, to 1e-15)
    got, rep = ft.ftsp2_train_coeffs_skip(0, beta0, mu0, L=L, nsamples=4000, iterations=8, accel=False)
    assert rep["accepted"] == sum(1 for h in hist if h[2])
    assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))
    assert abs(rep["cost"] - hist[-1][0]) <= 1e-6 * hist[-1][0]
    got_e, rep_e = ft.ftsp2_train_coeffs_skip(1, beta0, mu0, skip_init=got, nsamples=4000, iterations=4,
                                              accel=True, alpha=0.842704)
    ref_e = skipsp2.max_error(got_e, "entropy", beta0, mu0, alpha=0.842704, grid=4001)
    assert abs(rep_e["max_err"] - ref_e) < 0.5 * ref_e + 1e-9
