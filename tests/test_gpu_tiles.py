"""GPU parity of both tensor-core tile shapes (256 x 256 tiles on CTA pairs,
128 x 128 tiles on single CTAs) against the CPU oracle, and the tile-shape
autotuner (ftsp2_autotune / ftsp2_tile_shape / ftsp2_autotune_clear)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fermi, pipeline, rescale, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
# the bound of the main parity suite: 1e-6 for every mode
TOL_D = {"tf32x3": 1e-6, "bf16x3": 1e-6, "fp16x2": 1e-6}
TOL_S = 1e-6


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.fixture(scope="module")
def ms(ft):
    return ft.ModelSet()


def shape_flag(ft, shape):
    return ft.PAIR_TILES if shape == "pair" else ft.SINGLE_TILES


def solve(ft, ms, Hs, mus, kTs, mode, flags=0):
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=3, flags=flags)
    flat, _ = wl.pack_batch(Hs)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


def check(s, b, H, mu, kT, mode):
    ex = pipeline.method_exact(H, mu, kT, [PRINTED])
    rec = s.records()[b]
    assert rec["status"] == 0
    n = H.shape[0]
    D = s.matrix(b).double().cpu().numpy()
    assert np.max(np.abs(D - D.T)) == 0.0
    err = np.max(np.abs(D - ex["D"]))
    assert err < TOL_D[mode], (mode, n, err)
    tr = s.trace.cpu().numpy()[b]
    assert abs(tr[0] - np.trace(D)) < 1e-3
    assert abs(tr[1] - np.sum(D * D)) < 1e-3 * max(1.0, tr[1])
    S = float(s.S.cpu()[b])
    assert abs(S - ex["S"]) / n < TOL_S, (mode, n, S, ex["S"])


@pytest.mark.parametrize("shape", ["single", "pair"])
@pytest.mark.parametrize("n", [1, 3, 127, 128, 129, 255, 257, 300, 513])
def test_sizes_fp16x2(ft, ms, shape, n):
    # every edge of a 128 x 128 tile and of a 256 x 256 tile, plus tiny orders
    H = wl.chain_1d(n, 40 + n) if n > 1 else np.array([[0.25]])
    s = solve(ft, ms, [H], [0.1], [0.1], "fp16x2", shape_flag(ft, shape))
    check(s, 0, H, 0.1, 0.1, "fp16x2")


@pytest.mark.parametrize("shape", ["single", "pair"])
@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_other_modes(ft, ms, shape, mode):
    H = wl.chain_1d(300, 7)
    s = solve(ft, ms, [H], [-0.2], [0.15], mode, shape_flag(ft, shape))
    check(s, 0, H, -0.2, 0.15, mode)


@pytest.mark.parametrize("shape", ["single", "pair"])
def test_ragged_batch_both_chains(ft, ms, shape):
    # a ragged batch whose instances start at different global layers
    # (different beta') and straddle tile edges of both shapes
    ns = [64, 200, 129, 383, 96, 257]
    Hs = [wl.chain_1d(n, 50 + n) for n in ns]
    mus = [0.0, 0.3, -0.4, 0.1, 0.5, -0.1]
    kTs = [0.1, 0.3, 0.2, 0.1, 0.5, 0.15]
    s = solve(ft, ms, Hs, mus, kTs, "fp16x2", shape_flag(ft, shape))
    for b, H in enumerate(Hs):
        check(s, b, H, mus[b], kTs[b], "fp16x2")


def test_single_tiles_lattice_1024_and_refine(ft, ms):
    H = wl.lattice_3d((8, 8, 16), 0)
    kT = 0.1
    mu = fermi.mu_at_filling(np.linalg.eigvalsh(H), kT, 512)
    s = solve(ft, ms, [H], [mu], [kT], "fp16x2", ft.SINGLE_TILES | ft.REFINE2)
    check(s, 0, H, mu, kT, "fp16x2")


def test_shapes_agree(ft, ms):
    # the two shapes run the same K order per element; both stay within the
    # bound of each other that their separate bounds imply
    H = wl.lattice_3d((8, 8, 8), 3)
    a = solve(ft, ms, [H], [0.0], [0.1], "fp16x2", ft.SINGLE_TILES)
    b = solve(ft, ms, [H], [0.0], [0.1], "fp16x2", ft.PAIR_TILES)
    assert float((a.D - b.D).abs().max()) < 2 * TOL_D["fp16x2"]
    assert abs(float(a.S[0]) - float(b.S[0])) / 512 < 2 * TOL_S


def test_autotune_records_and_reuses_choice(ft, ms):
    ft.ftsp2_autotune_clear()
    ns = [96, 160, 320, 250]
    Hs = [wl.chain_1d(n, 60 + n) for n in ns]
    mus, kTs = [0.0, 0.2, -0.1, 0.3], [0.1, 0.2, 0.15, 0.3]
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    s = ft.Solver(ns, mus, kTs, ms, mode="fp16x2", want=3)
    shape0, tuned0 = s.tile_shape()
    assert shape0 in (0, 1) and not tuned0
    choice, ms_single, ms_pair = s.autotune(Hd, reps=2)
    assert choice in (0, 1)
    assert ms_single > 0 and ms_pair > 0
    assert choice == (1 if ms_pair <= ms_single else 0)
    assert s.tile_shape() == (choice, True)
    # the same signature in another order of instances reuses the record
    s2 = ft.Solver(ns[::-1], mus[::-1], kTs[::-1], ms, mode="fp16x2", want=3)
    assert s2.tile_shape() == (choice, True)
    # a forcing flag wins over the record
    forced = ft.Solver(ns, mus, kTs, ms, mode="fp16x2", want=3,
                       flags=ft.SINGLE_TILES if choice else ft.PAIR_TILES)
    assert forced.tile_shape() == (1 - choice, False)
    # the tuned default reproduces the forced run of the chosen shape bit for bit
    s.run(Hd, sync=True)
    ref = ft.Solver(ns, mus, kTs, ms, mode="fp16x2", want=3,
                    flags=ft.PAIR_TILES if choice else ft.SINGLE_TILES)
    ref.run(Hd, sync=True)
    torch.cuda.synchronize()
    assert torch.equal(s.D, ref.D) and torch.equal(s.S, ref.S) and torch.equal(s.trace, ref.trace)
    for b, H in enumerate(Hs):
        check(s, b, H, mus[b], kTs[b], "fp16x2")
    ft.ftsp2_autotune_clear()
    assert s.tile_shape()[1] is False


def test_autotune_fp32_mode_has_no_shape(ft, ms):
    H = wl.chain_1d(130, 3)
    s = ft.Solver([130], [0.0], [0.1], ms, mode="fp32", want=3)
    choice, a, b = s.autotune(torch.from_numpy(H.ravel().copy()).cuda(), reps=1)
    assert choice == -1 and a == 0.0 and b == 0.0
    assert s.tile_shape() == (-1, False)
