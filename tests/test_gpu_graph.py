"""The hot path recorded into a CUDA graph (stream capture through the C ABI)
and replayed: same results as eager runs, new inputs picked up on replay."""
import numpy as np
import pytest

import workloads as wl
from oracle import pipeline, rescale, tables

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


@pytest.mark.parametrize("mode,flags", [("fp16x2", 0), ("bf16x3", "REFINE2"), ("fp32", 0)])
def test_graph_replay_matches_eager(ft, mode, flags):
    ms = ft.ModelSet()
    ns = [200, 130, 257]
    mus, kTs = [0.1, -0.2, 0.0], [0.1, 0.2, 0.15]
    fl = getattr(ft, flags) if flags else 0
    Hs = [wl.chain_1d(n, 70 + n) for n in ns]
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    eager = ft.Solver(ns, mus, kTs, ms, mode=mode, want=3, flags=fl)
    eager.run(Hd, sync=True)
    s = ft.Solver(ns, mus, kTs, ms, mode=mode, want=3, flags=fl)
    g = s.graph(Hd)
    s.D.zero_()
    s.S.zero_()
    s.trace.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(s.D, eager.D) and torch.equal(s.S, eager.S) and torch.equal(s.trace, eager.trace)
    # new Hamiltonians in the same buffer and new mu: the replay follows them
    Hs2 = [wl.chain_1d(n, 90 + n) for n in ns]
    flat2, _ = wl.pack_batch(Hs2)
    Hd.copy_(torch.from_numpy(flat2))
    mus2 = [0.3, 0.0, -0.1]
    s.set_mu_kT(mus2, kTs)
    g.replay()
    torch.cuda.synchronize()
    tol = 1e-6
    for b, H in enumerate(Hs2):
        ex = pipeline.method_exact(H, mus2[b], kTs[b], [PRINTED])
        assert s.records()[b]["status"] == 0
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - ex["D"])) < tol
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6


def test_sync_flag_refused_while_capturing(ft):
    ms = ft.ModelSet()
    H = wl.chain_1d(100, 1)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    s = ft.Solver([100], [0.0], [0.1], ms, mode="fp16x2", want=3)
    s.run(Hd)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(ft.Ftsp2Error):
        with torch.cuda.graph(g):
            s.run(Hd, sync=True)
