"""Bounded device-side waits of the multi-layer launches.

A multi-layer launch runs consecutive layers as (layer, tile) work items, and
an item waits until every tile of the previous layer of its chain has
finished.  The test hook ftsp2_debug_stall_layer makes the items of one layer
wait for one completion more than can ever arrive (a flag that nothing sets),
with a short wait limit (ftsp2_set_wait_limit_ns).  The call must end on its
own with FTSP2_E_TIMEOUT in every record, promptly, and the next ordinary call
in the same process must succeed and reproduce an undisturbed run bit for bit
(the context stays usable and nothing of the failed call leaks into the next).
No GPU fault is involved: the wait runs out, records the status and the
kernel finishes its work list without loads, MMAs or stores."""
import time

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

E_TIMEOUT = -6


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.mark.parametrize("shape", ["pair", "pair_deferred", "single"])
def test_stalled_dependency_ends_in_timeout(ft, shape):
    flags = {"pair": ft.PAIR_TILES | ft.EPI_INLINE, "pair_deferred": ft.PAIR_TILES | ft.EPI_DEFERRED,
             "single": ft.SINGLE_TILES}[shape]
    H = wl.lattice_3d((8, 8, 16), 0)
    n = H.shape[0]
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    s = ft.Solver([n], [0.0], [0.1], ft.ModelSet(), mode="fp16x2", want=3, flags=flags)
    c0 = ft.kernel_launch_count()
    assert s.run(Hd, sync=True) == 0
    multi = ft.kernel_launch_count() - c0
    per_layer = ft.Solver([n], [0.0], [0.1], ft.ModelSet(), mode="fp16x2", want=3, flags=flags | ft.LAYER_LAUNCHES)
    c0 = ft.kernel_launch_count()
    assert per_layer.run(Hd, sync=True) == 0
    if multi >= ft.kernel_launch_count() - c0:
        pytest.skip("multi-layer launches are not available on this device")
    D0, S0, T0 = s.D.clone(), s.S.clone(), s.trace.clone()

    default = ft.wait_limit_ns()
    ft.set_wait_limit_ns(2_000_000)            # 2 ms
    ft.debug_stall_layer(5)
    try:
        t0 = time.perf_counter()
        st = s.run(Hd, sync=True)
        dt = time.perf_counter() - t0
    finally:
        ft.debug_stall_layer(-1)
        ft.set_wait_limit_ns(default)
    assert st == E_TIMEOUT, ft.status_string(st)
    assert np.all(s.records()["status"] == E_TIMEOUT)
    assert dt < 5.0, dt

    # the next ordinary call succeeds and matches the undisturbed run
    assert ft.wait_limit_ns() == default
    assert s.run(Hd, sync=True) == 0
    assert torch.equal(s.D, D0) and torch.equal(s.S, S0) and torch.equal(s.trace, T0)
