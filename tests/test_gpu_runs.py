"""GPU parity of multi-layer launches: consecutive layers of the main format
run in one persistent cooperative launch whose work items are (layer, tile)
and whose items wait for the previous layer of their chain through device
counters.  The arithmetic per tile is unchanged, so D, S and the traces must
equal those of one launch per layer (FTSP2_LAYER_LAUNCHES) bit for bit, with
fewer kernel launches; and the oracle."""
import glob
import os

import numpy as np
import pytest

import workloads as wl
from oracle import pipeline, rescale, tables

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
TABLES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_08523_gb300", "tables")


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


def solve(ft, Hs, mus, kTs, ms, mode, flags):
    flat, _ = wl.pack_batch(Hs)
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=3, flags=flags)
    Hd = torch.from_numpy(flat).cuda()
    s.run(Hd, sync=True)                      # first run: tile-shape records, attributes
    torch.cuda.synchronize()
    n0 = ft.kernel_launch_count()
    s.run(Hd, sync=True)
    torch.cuda.synchronize()
    return s, ft.kernel_launch_count() - n0


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("shape", ["pair", "single"])
@pytest.mark.parametrize("extra", ["", "inline", "refine_tc", "refine_fp32", "full"])
def test_runs_bit_identical_to_layer_launches(ft, mode, shape, extra):
    if extra == "refine_tc" and mode == "bf16x3":
        pytest.skip("no refinement layers on BF16X3")
    Hs = [wl.lattice_3d((8, 8, 16), 3), wl.chain_1d(700, 8), wl.chain_1d(129, 9)]
    mus, kTs = [0.0, 0.2, -0.1], [0.1, 0.1, 0.2]
    f = ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES
    f |= {"": 0, "inline": ft.EPI_INLINE, "refine_tc": ft.REFINE2 | ft.REFINE_TC, "refine_fp32": ft.REFINE2,
          "full": ft.FULL_OPERANDS}[extra]
    a, la = solve(ft, Hs, mus, kTs, ft.ModelSet(), mode, f)
    b, lb = solve(ft, Hs, mus, kTs, ft.ModelSet(), mode, f | ft.LAYER_LAUNCHES)
    assert la < lb, (la, lb)                  # the layers ran in fewer launches
    assert torch.equal(a.D, b.D) and torch.equal(a.S, b.S) and torch.equal(a.trace, b.trace)
    assert all(int(r["status"]) == 0 for r in a.records())
    for i, H in enumerate(Hs):
        ex = pipeline.method_exact(H, mus[i], kTs[i], [PRINTED])
        D = a.matrix(i).double().cpu().numpy()
        assert np.max(np.abs(D - ex["D"])) < 1e-6, (mode, shape, extra, i)


@pytest.mark.parametrize("shape", ["pair", "single"])
def test_runs_with_late_starting_models(ft, shape):
    # instances whose models have fewer layers start at later global layers:
    # their tiles are inactive items in the run's first layers
    paths = [os.path.join(TABLES, "entropy_b1500_L26.json")]
    paths += sorted(p for p in glob.glob(os.path.join(TABLES, "b*.json"))
                    if int(os.path.basename(p)[1:].split("_")[0]) >= 3000)
    ms = ft.ModelSet.from_json(paths)
    batch = wl.ragged_batch(16, 5)
    Hs = [b["H"] for b in batch]
    mus, kTs = [b["mu"] for b in batch], [b["kT"] for b in batch]
    f = ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES
    a, la = solve(ft, Hs, mus, kTs, ms, "fp16x2", f)
    b, lb = solve(ft, Hs, mus, kTs, ms, "fp16x2", f | ft.LAYER_LAUNCHES)
    models = {int(r["model"]) for r in a.records() if r["status"] == 0}
    assert len(models) >= 2, models
    assert la < lb, (la, lb)
    assert torch.equal(a.D, b.D) and torch.equal(a.S, b.S) and torch.equal(a.trace, b.trace)


def test_runs_repeat_identically(ft):
    # the device counters are reset by every solve; repeated solves and a
    # CUDA-graph replay give the same bits
    Hs = [wl.lattice_3d((8, 16, 16), 1)]
    s = ft.Solver([Hs[0].shape[0]], [0.0], [0.1], ft.ModelSet(), mode="fp16x2", want=3, flags=ft.PAIR_TILES)
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    s.run(Hd, sync=True)
    D0, S0 = s.D.clone(), s.S.clone()
    for _ in range(3):
        s.run(Hd)
    torch.cuda.synchronize()
    assert torch.equal(s.D, D0) and torch.equal(s.S, S0)
    g = s.graph(Hd)
    s.D.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(s.D, D0) and torch.equal(s.S, S0)
