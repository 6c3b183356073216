"""ftsp2_density_noalloc: the density entry point for callers that cannot
allocate device memory (graph capture in progress, host applications that own
all device memory, loops that must not pay for cudaMalloc).  It takes its
scratch from a fixed 8 MiB array inside the library instead of a caller
workspace.  Checked through the C ABI against ftsp2_density on the same inputs,
on two calls in a row (the array keeps the previous call's contents), and for
the size limit.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


def _inputs(ft, Hs, mus, kTs):
    from paper_2605_08523_gb300 import INST_DTYPE, _instances
    host, offs, total = _instances([H.shape[0] for H in Hs], mus, kTs)
    raw = np.frombuffer(bytes(host), dtype=np.uint8).copy()
    d_inst = torch.from_numpy(raw).cuda()
    flat, _ = wl.pack_batch(Hs)
    return host, d_inst, torch.from_numpy(flat).cuda(), total


def _p(t):
    return C.c_void_p(t.data_ptr())


def _run_noalloc(ft, ms, host, d_inst, Hd, nb, total, mode):
    D = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    tr = torch.full((nb, 2), float("nan"), dtype=torch.float64, device="cuda")
    rec = torch.zeros(nb * 64, dtype=torch.uint8, device="cuda")
    st = ft.lib().ftsp2_density_noalloc(_p(Hd), host, _p(d_inst), nb, ms.handle, ft.MODES[mode], 0, _p(D), _p(tr),
                                        _p(rec), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, D, tr, rec.cpu().numpy().view(ft.REC_DTYPE)


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
def test_noalloc_matches_workspace_entry_point(ft, mode):
    ms = ft.ModelSet()
    Hs = [wl.chain_1d(n, 40 + n) for n in (64, 100, 150)]
    mus, kTs = [0.0, 0.2, -0.1], [0.1, 0.15, 0.2]
    host, d_inst, Hd, total = _inputs(ft, Hs, mus, kTs)
    ref = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=1)
    ref.run(Hd, sync=True)
    for call in range(2):            # two calls in a row on the same static scratch
        st, D, tr, rec = _run_noalloc(ft, ms, host, d_inst, Hd, len(Hs), total, mode)
        assert st == 0, ft.status_string(st)
        assert np.all(rec["status"] == 0)
        # same kernels, same inputs: within the parity tolerance (here bitwise)
        assert torch.max(torch.abs(D - ref.D)).item() <= 8e-6
        assert torch.equal(D, ref.D)
        assert torch.allclose(tr, ref.trace, rtol=0, atol=1e-9)


def test_noalloc_single_instance_largest_supported(ft):
    ms = ft.ModelSet()
    H = wl.chain_1d(512, 3)
    host, d_inst, Hd, total = _inputs(ft, [H], [0.0], [0.1])
    ref = ft.Solver([512], [0.0], [0.1], ms, mode="fp16x2", want=1)
    ref.run(Hd, sync=True)
    for call in range(2):
        st, D, tr, rec = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp16x2")
        assert st == 0
        assert torch.equal(D, ref.D)


def test_noalloc_rejects_oversize_and_sync(ft):
    ms = ft.ModelSet()
    n = 1024
    H = np.eye(n)
    host, d_inst, Hd, total = _inputs(ft, [H], [0.5], [0.1])
    st, D, _, _ = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp16x2")
    assert st == ft._lib.E_WORKSPACE
    assert torch.isnan(D).all()                 # nothing was launched
    rec = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = ft.lib().ftsp2_density_noalloc(_p(Hd), host, _p(d_inst), 1, ms.handle, ft.FP16X2, ft.SYNC, _p(D), None,
                                        _p(rec), None)
    assert st == ft._lib.E_ARG
