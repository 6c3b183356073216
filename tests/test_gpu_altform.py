"""GPU parity of tables of the one-term form (Eq. mlsp2_alt): a model set built
from such tables (converted by ftsp2_alt_to_mlsp2) runs the layer kernels and
matches the oracle's one-term recursion on the eigenvalues; and the library's
training in this form against the oracle's."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import altform, fermi, train

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    with open(os.path.join(ROOT, "tests", "golden", "alt_table.json")) as f:
        return json.load(f)


def model_set(ft, d):
    return ft.ModelSet([dict(alt=d["alt"], alt_entropy=d["alt_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                             alpha=d["alpha"])])


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("shape", ["pair", "single"])
def test_one_term_tables_match_oracle(ft, golden, mode, shape):
    d = golden
    ms = model_set(ft, d)
    Hs = [wl.chain_1d(300, 4), wl.lattice_3d((8, 8, 8), 2)]
    ns = [H.shape[0] for H in Hs]
    kTs = [0.2, 0.3]
    mus = [0.1, -0.2]
    flat, _ = wl.pack_batch(Hs)
    flags = ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES
    s = ft.Solver(ns, mus, kTs, ms, mode=mode, want=3, flags=flags)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    for b, H in enumerate(Hs):
        ex = altform.method_exact(H, mus[b], kTs[b], d["alt"], d["beta0"], d["mu0"], d["alpha"], d["alt_entropy"])
        assert ex["D"] is not None, "instance outside the table's region"
        assert s.records()[b]["status"] == 0
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - ex["D"])) < 1e-6, (mode, b)
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / ns[b] < 1e-6
        # and against the eigendecomposition within the table's fit error
        Dref, Sref, _, _ = fermi.eig_reference(H, mus[b], kTs[b])
        assert np.max(np.abs(D - Dref)) < d["max_err"] + 1e-6


def test_training_in_one_term_form_matches_oracle(ft):
    # a few LM iterations from the SP2 sequence: the library's chain rule on the
    # GPU reductions and the oracle's Jacobian give the same steps
    beta0, mu0, L = 60.0, 1.0 / 3.0, 12
    x = train.sample_grid(4000, beta0, mu0)
    a0 = altform.sp2_alt(mu0, L)
    ref, hist = altform.lm_fit(a0, x, "fermi", beta0, mu0, iters=8, accel=False)
    # the library's own samples and start (nsamples = 4000, seed 0, no start
    # table: ftsp2_train_init_alt) are the oracle's, to 1e-15 (tests/test_train_inputs.py)
    got, rep = ft.ftsp2_train_coeffs_alt(0, beta0, mu0, L=L, nsamples=4000, iterations=8, accel=False)
    assert rep["accepted"] == sum(1 for h in hist if h[2])
    assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))
    assert abs(rep["cost"] - hist[-1][0]) <= 1e-6 * hist[-1][0]
    # with geodesic acceleration the cost falls at least as far as without
    got_a, rep_a = ft.ftsp2_train_coeffs_alt(0, beta0, mu0, alt_init=a0, nsamples=4000, iterations=8, accel=True)
    assert rep_a["cost"] <= 1.05 * rep["cost"]
    assert abs(rep_a["max_err"] - altform.max_error(got_a, "fermi", beta0, mu0, grid=4001)) < 0.5 * rep_a["max_err"] + 1e-9
