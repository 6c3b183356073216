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


@pytest.mark.parametrize("n", [512, 640])
def test_noalloc_single_instance_up_to_the_limit(ft, n):
    # n = 640 is the largest FP16X2 instance the 8 MiB array holds
    ms = ft.ModelSet()
    H = wl.chain_1d(n, 3)
    host, d_inst, Hd, total = _inputs(ft, [H], [0.0], [0.1])
    ref = ft.Solver([n], [0.0], [0.1], ms, mode="fp16x2", want=1)
    ref.run(Hd, sync=True)
    for call in range(2):
        st, D, tr, rec = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp16x2")
        assert st == 0
        assert torch.equal(D, ref.D)


@pytest.mark.parametrize("n", [641, 1024])
def test_noalloc_rejects_oversize_and_sync(ft, n):
    # n = 641 pads to 768 and needs more than the array: refused before any launch
    ms = ft.ModelSet()
    H = np.eye(n)
    host, d_inst, Hd, total = _inputs(ft, [H], [0.5], [0.1])
    st, D, _, _ = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp16x2")
    assert st == ft._lib.E_WORKSPACE
    assert torch.isnan(D).all()                 # nothing was launched
    rec = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = ft.lib().ftsp2_density_noalloc(_p(Hd), host, _p(d_inst), 1, ms.handle, ft.FP16X2, ft.SYNC, _p(D), None,
                                        _p(rec), None)
    assert st == ft._lib.E_ARG


_FIRST_CALL_WHILE_CAPTURING = r"""
import ctypes as C, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2605_08523_gb300 as ft
import workloads as wl
from paper_2605_08523_gb300 import _instances
ms = ft.ModelSet()
H = wl.chain_1d(128, 5)
host, _, _ = _instances([128], [0.0], [0.1])
d_inst = torch.from_numpy(np.frombuffer(bytes(host), dtype=np.uint8).copy()).cuda()
Hd = torch.from_numpy(H.ravel().copy()).cuda()
D = torch.full((128 * 128,), float("nan"), dtype=torch.float32, device="cuda")
rec = torch.zeros(64, dtype=torch.uint8, device="cuda")
p = lambda t: C.c_void_p(t.data_ptr())
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    st_cap = ft.lib().ftsp2_density_noalloc(p(Hd), host, p(d_inst), 1, ms.handle, ft.FP16X2, 0, p(D), None, p(rec),
                                            C.c_void_p(s.cuda_stream))
untouched = bool(torch.isnan(D).all())
st = ft.lib().ftsp2_density_noalloc(p(Hd), host, p(d_inst), 1, ms.handle, ft.FP16X2, 0, p(D), None, p(rec),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
torch.cuda.synchronize()
print(json.dumps({"st_cap": st_cap, "untouched": untouched, "st": st, "finite": bool(torch.isfinite(D).all())}))
"""


def test_noalloc_first_call_while_capturing_is_refused(ft, tmp_path):
    # In a fresh process the array's address is not known yet: a first call
    # made while the stream is being captured is refused before the lookup
    # (which could load the module inside the capture), and the next ordinary
    # call works.
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    prog = tmp_path / "first_call.py"
    prog.write_text(_FIRST_CALL_WHILE_CAPTURING)
    r = subprocess.run([sys.executable, str(prog), root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["st_cap"] == ft._lib.E_ARG and out["untouched"]
    assert out["st"] == 0 and out["finite"]


def test_noalloc_max_sp2_set(ft):
    # a Max-SP2 table (FP32 mode; 13 state planes per chain) through the
    # allocation-free entry: the same result as the workspace entry point; the
    # tensor-core modes refuse such a set
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "tests", "golden", "max_table.json")) as f:
        d = json.load(f)
    ms = ft.ModelSet([dict(max=d["max"], max_entropy=d["max_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                           alpha=d["alpha"])])
    H = wl.chain_1d(96, 4)
    host, d_inst, Hd, total = _inputs(ft, [H], [0.05], [0.3])
    ref = ft.Solver([96], [0.05], [0.3], ms, mode="fp32", want=1)
    ref.run(Hd, sync=True)
    st, D, tr, rec = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp32")
    assert st == 0, ft.status_string(st)
    assert torch.equal(D, ref.D)
    st, _, _, _ = _run_noalloc(ft, ms, host, d_inst, Hd, 1, total, "fp16x2")
    assert st == ft._lib.E_UNSUPPORTED
