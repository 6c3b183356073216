"""The reference computations bench.py makes on the GPU (FP64 torch), pinned to
the oracle: the eigendecomposition references D_ref, S_ref and the half-filling
mu (bench.eig_reference_gpu), and the method-exact D_rec, S_rec that isolate
the library's rounding (bench.method_exact_gpu, from the library's rescale
records).  The bench's accuracy figures rest on these two functions."""
import numpy as np
import pytest

import workloads as wl
from oracle import fermi, pipeline, rescale, tables

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


def test_eig_reference_gpu_matches_oracle(ft):
    import bench
    H = wl.lattice_3d((8, 8, 8), 3)
    n, kT = H.shape[0], 0.1
    mu, D, S, eps, V = bench.eig_reference_gpu(torch.from_numpy(H).cuda(), kT, n)
    mu_o = fermi.mu_at_filling(np.linalg.eigvalsh(H), kT, n / 2)
    D_o, S_o, tr_o, _ = fermi.eig_reference(H, mu_o, kT)
    assert abs(mu - mu_o) < 1e-9
    assert np.max(np.abs(D.cpu().numpy() - D_o)) < 1e-11
    assert abs(S - S_o) < 1e-9 * n
    # with mu given
    mu2, D2, S2, _, _ = bench.eig_reference_gpu(torch.from_numpy(H).cuda(), 0.2, n, mu=0.3)
    D2_o, S2_o, _, _ = fermi.eig_reference(H, 0.3, 0.2)
    assert mu2 == 0.3 and np.max(np.abs(D2.cpu().numpy() - D2_o)) < 1e-11 and abs(S2 - S2_o) < 1e-9 * n


@pytest.mark.parametrize("where", ["top", "half", "bottom"])
def test_method_exact_gpu_matches_oracle(ft, where):
    import bench
    H = wl.lattice_3d((8, 8, 8), 5)
    n, kT = H.shape[0], 0.1
    eps_np = np.linalg.eigvalsh(H)
    # mu near the top of the spectrum (mu' < 1/2: no flip), at half filling,
    # or near the bottom (mu' > 1/2: Eq. flip)
    mu = {"top": float(eps_np[-20]), "half": fermi.mu_at_filling(eps_np, kT, n / 2),
          "bottom": float(eps_np[20])}[where]
    s = ft.Solver([n], [mu], [kT], ft.ModelSet(), mode="fp16x2", want=3)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    assert s.run(Hd, sync=True) == 0
    rec = s.records()[0]
    eps, V = torch.linalg.eigh(Hd.view(n, n))
    table = {"theta": [tuple(r) for r in tables.PRINTED_B1500], "mu0": 1.0 / 3.0, "alpha": PRINTED.alpha,
             "theta_entropy": None}
    Drec, Srec = bench.method_exact_gpu(eps, V, rec, table, mu)
    ex = pipeline.method_exact(H, mu, kT, [PRINTED])
    assert bool(rec["flip"]) == ex["rec"].flip
    if where != "half":
        assert ex["rec"].flip == (where == "bottom")
    assert np.max(np.abs(Drec.cpu().numpy() - ex["D"])) < 1e-9
    assert abs(Srec - ex["S"]) < 1e-8 * n
