"""GPU parity of the deferred final epilogue of the 256 x 256 pair tiles
(FTSP2_EPI_DEFERRED: store warps write Z_{k+1}, A_{k+1} and the next operands
from a per-CTA scratch while the next tile accumulates) against the CPU oracle,
and bit-for-bit against the inline epilogue (FTSP2_EPI_INLINE): both run the
same accumulation and the same epilogue arithmetic."""
import numpy as np
import pytest

import workloads as wl
from oracle import fermi, pipeline, rescale, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
TOL_D = 1e-6
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


def solve(ft, ms, Hs, mus, kTs, mode, flags):
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=3, flags=flags)
    flat, _ = wl.pack_batch(Hs)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


def both(ft, ms, Hs, mus, kTs, mode="fp16x2", extra=0):
    d = solve(ft, ms, Hs, mus, kTs, mode, ft.PAIR_TILES | ft.EPI_DEFERRED | extra)
    i = solve(ft, ms, Hs, mus, kTs, mode, ft.PAIR_TILES | ft.EPI_INLINE | extra)
    assert torch.equal(d.D, i.D), "deferred and inline epilogues differ"
    assert torch.equal(d.S, i.S) and torch.equal(d.trace, i.trace)
    assert np.array_equal(d.records()["status"], i.records()["status"])
    return d


def check(s, b, H, mu, kT):
    ex = pipeline.method_exact(H, mu, kT, [PRINTED])
    assert s.records()[b]["status"] == 0
    n = H.shape[0]
    D = s.matrix(b).double().cpu().numpy()
    assert np.max(np.abs(D - D.T)) == 0.0
    err = np.max(np.abs(D - ex["D"]))
    assert err < TOL_D, (n, err)
    S = float(s.S.cpu()[b])
    assert abs(S - ex["S"]) / n < TOL_S, (n, S, ex["S"])


@pytest.mark.parametrize("n", [1, 3, 129, 255, 256, 257, 300, 513, 700])
def test_sizes_match_oracle_and_inline(ft, ms, n):
    # tile edges of the pair shape (256), the order beyond the padded pitch
    # (n = 300: pitch 384, the second column tile ends at 512), tiny orders
    H = wl.chain_1d(n, 70 + n) if n > 1 else np.array([[0.25]])
    s = both(ft, ms, [H], [0.1], [0.1])
    check(s, 0, H, 0.1, 0.1)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_other_modes(ft, ms, mode):
    H = wl.chain_1d(513, 9)
    s = both(ft, ms, [H], [-0.2], [0.15], mode)
    check(s, 0, H, -0.2, 0.15)


def test_ragged_batch(ft, ms):
    # instances that start at different global layers and straddle the pair
    # tile edges; each CTA's scratch serves tiles of several instances
    ns = [64, 200, 129, 383, 96, 257, 511]
    Hs = [wl.chain_1d(n, 80 + n) for n in ns]
    mus = [0.0, 0.3, -0.4, 0.1, 0.5, -0.1, 0.2]
    kTs = [0.1, 0.3, 0.2, 0.1, 0.5, 0.15, 0.1]
    s = both(ft, ms, Hs, mus, kTs)
    for b, H in enumerate(Hs):
        check(s, b, H, mus[b], kTs[b])


def test_lattice_1024_with_tensor_core_refinement(ft, ms):
    # more tiles than CTA pairs (each pair runs several tiles through the
    # scratch); the BF16X3 refinement layers run deferred as well
    H = wl.lattice_3d((8, 8, 16), 1)
    kT = 0.1
    mu = fermi.mu_at_filling(np.linalg.eigvalsh(H), kT, 512)
    s = both(ft, ms, [H], [mu], [kT], extra=ft.REFINE2 | ft.REFINE_TC)
    check(s, 0, H, mu, kT)


def test_default_is_bit_identical_to_forced_choice(ft, ms):
    # the default picks one of the two epilogues; either way the result is the
    # forced runs' result
    H = wl.lattice_3d((8, 8, 8), 5)
    d = solve(ft, ms, [H], [0.0], [0.1], "fp16x2", ft.PAIR_TILES)
    f = solve(ft, ms, [H], [0.0], [0.1], "fp16x2", ft.PAIR_TILES | ft.EPI_DEFERRED)
    assert torch.equal(d.D, f.D) and torch.equal(d.S, f.S)
