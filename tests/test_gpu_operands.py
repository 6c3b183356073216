"""GPU parity of the upper-triangle operand storage (default for FP16X2 and
BF16X3 layers): K-slices left of a panel's diagonal block are loaded as
transposed panels (MN-major tcgen05 operands) instead of from a stored mirror.
The tensor cores see the same operand values, so the results must equal those
of full operand matrices (FTSP2_FULL_OPERANDS) bit for bit; and the oracle."""
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


def solve(ft, Hs, mus, kTs, mode, flags):
    flat, _ = wl.pack_batch(Hs)
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ft.ModelSet(), mode=mode, want=3, flags=flags)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
@pytest.mark.parametrize("shape", ["pair", "single"])
@pytest.mark.parametrize("extra", ["", "deferred", "refine_tc", "refine_fp32"])
def test_upper_triangle_operands_bit_identical(ft, mode, shape, extra):
    if extra == "deferred" and shape == "single":
        pytest.skip("the deferred epilogue runs on pair tiles")
    Hs = [wl.lattice_3d((8, 8, 16), 3), wl.chain_1d(700, 8), wl.chain_1d(129, 9)]
    mus, kTs = [0.0, 0.2, -0.1], [0.1, 0.1, 0.2]
    f = ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES
    f |= {"": 0, "deferred": ft.EPI_DEFERRED, "refine_tc": ft.REFINE2 | ft.REFINE_TC,
          "refine_fp32": ft.REFINE2}[extra]
    a = solve(ft, Hs, mus, kTs, mode, f)
    b = solve(ft, Hs, mus, kTs, mode, f | ft.FULL_OPERANDS)
    assert torch.equal(a.D, b.D) and torch.equal(a.S, b.S) and torch.equal(a.trace, b.trace)
    for i, H in enumerate(Hs):
        ex = pipeline.method_exact(H, mus[i], kTs[i], [PRINTED])
        D = a.matrix(i).double().cpu().numpy()
        assert np.max(np.abs(D - D.T)) == 0.0
        assert np.max(np.abs(D - ex["D"])) < 1e-6, (mode, shape, extra, i)
        assert abs(float(a.S.cpu()[i]) - ex["S"]) / H.shape[0] < 1e-6


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
@pytest.mark.parametrize("shape", ["pair", "single"])
def test_late_starting_models_bit_identical(ft, mode, shape):
    # models with fewer layers start at later global layers: their layer-0
    # operands, written by init as the upper triangle plus the diagonal blocks,
    # are first read by a launch in the middle of the sequence
    import glob
    import os
    tdir = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_08523_gb300",
                        "tables")
    paths = [os.path.join(tdir, "entropy_b1500_L26.json")]
    paths += sorted(p for p in glob.glob(os.path.join(tdir, "b*.json"))
                    if int(os.path.basename(p)[1:].split("_")[0]) >= 3000)
    ms = ft.ModelSet.from_json(paths)
    batch = wl.ragged_batch(16, 5)
    Hs = [b["H"] for b in batch]
    mus, kTs = [b["mu"] for b in batch], [b["kT"] for b in batch]
    f = ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES
    flat, _ = wl.pack_batch(Hs)
    out = []
    for extra in (0, ft.FULL_OPERANDS):
        s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=3, flags=f | extra)
        s.run(torch.from_numpy(flat).cuda(), sync=True)
        torch.cuda.synchronize()
        out.append(s)
    a, b = out
    models = {int(r["model"]) for r in a.records() if r["status"] == 0}
    assert len(models) >= 2, models          # more than one start layer in the batch
    assert torch.equal(a.D, b.D) and torch.equal(a.S, b.S) and torch.equal(a.trace, b.trace)
