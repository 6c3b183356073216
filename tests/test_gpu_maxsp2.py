"""GPU parity of Max-SP2 tables (FTSP2_FAMILY_MAX, FP32 mode: every stored
layer kept as an FP32 state plane) against the oracle's Max-SP2 recursion on
the eigenvalues: the golden trained tables (a Max-SP2 table and a Skip-SP2
table with two stored layers and two accumulators, run through the library's
embedding ftsp2_skip_to_max), the embedded one-accumulator golden table
against the Skip-SP2 path, a ragged batch mixing Max-SP2 and Eq. mlsp2
tables, the workspace sizing, and the modes that refuse such tables."""
import ctypes as C
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import fermi, maxsp2, skipsp2, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# FP32 products over n terms and up to 20 stored layers; the bar of every
# other FP32-class path
TOL_D = 1e-6


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
    with open(os.path.join(ROOT, "tests", "golden", "max_table.json")) as f:
        return json.load(f)


def run(ft, ms, Hs, mus, kTs, mode="fp32", want=3, flags=0):
    flat, _ = wl.pack_batch(Hs)
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=want, flags=flags)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


def max_set(ft, d, key="max", key_e="max_entropy"):
    return ft.ModelSet([dict(max=d[key], max_entropy=d[key_e], beta0=d["beta0"], mu0=d["mu0"], alpha=d["alpha"])])


def check(ft, s, Hs, mus, kTs, p, L, d, pe, Le):
    for b, H in enumerate(Hs):
        ex = maxsp2.method_exact(H, mus[b], kTs[b], p, L, d["beta0"], d["mu0"], d["alpha"], pe, Le)
        assert ex["D"] is not None
        assert s.records()[b]["status"] == 0
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - D.T)) == 0.0
        err = np.max(np.abs(D - ex["D"]))
        assert err < TOL_D, (b, err)
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6
        tr = s.trace.cpu().numpy()[b]
        assert abs(tr[0] - ex["trD"]) / H.shape[0] < 1e-6


def test_max_table_matches_oracle(ft, golden):
    d = golden
    Hs = [wl.chain_1d(300, 4), wl.lattice_3d((8, 8, 8), 2), wl.chain_1d(77, 9)]
    mus, kTs = [0.1, -0.2, 0.0], [0.2, 0.3, 0.25]
    s = run(ft, max_set(ft, d), Hs, mus, kTs)
    check(ft, s, Hs, mus, kTs, d["max"], d["L"], d, d["max_entropy"], d["L"])
    # and the density against the exact Fermi operator within the table's own error
    Dref, _, _, _ = fermi.eig_reference(Hs[0], mus[0], kTs[0])
    assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - Dref)) < d["max_err"] + 1e-6


def test_skip_two_layers_two_accumulators_through_the_library_embedding(ft, golden):
    d = golden
    t = d["skip22"]
    p = ft.ftsp2_skip_to_max(t["alpha"], t["beta"], t["gamma"], t["A0"], t["gL"])
    assert np.max(np.abs(p - maxsp2.skip_to_max({k: np.array(v) for k, v in t.items()}))) < 1e-12
    Ls = np.array(t["alpha"]).shape[0]
    ms = ft.ModelSet([dict(max=p, beta0=d["beta0"], mu0=d["mu0"], alpha=d["alpha"])])
    Hs = [wl.lattice_3d((8, 8, 8), 5), wl.chain_1d(200, 1)]
    mus, kTs = [0.05, 0.3], [0.3, 0.2]
    s = run(ft, ms, Hs, mus, kTs)
    check(ft, s, Hs, mus, kTs, p, Ls, d, p, Ls)
    # the Skip-SP2 recursion itself gives the same density
    ex = maxsp2.method_exact(Hs[0], mus[0], kTs[0], p, Ls, d["beta0"], d["mu0"], d["alpha"])
    eps, V = np.linalg.eigh(Hs[0])
    f = maxsp2.skip_scalar(ex["x0"], {k: np.array(v) for k, v in t.items()})
    if ex["rec"].flip:
        f = 1.0 - f
    assert np.max(np.abs((V * f) @ V.T - ex["D"])) < 1e-10


def test_embedded_one_accumulator_table(ft):
    with open(os.path.join(ROOT, "tests", "golden", "skip_table.json")) as f:
        d = json.load(f)
    p = maxsp2.skip1_to_max(np.array(d["skip"]))
    pe = maxsp2.skip1_to_max(np.array(d["skip_entropy"]))
    L = d["L"]
    H = wl.lattice_3d((8, 8, 8), 6)
    mu, kT = 0.0, 0.4                  # beta' inside the beta0 = 100 table's region
    ex = skipsp2.method_exact(H, mu, kT, d["skip"], d["beta0"], d["mu0"], d["alpha"], d["skip_entropy"])
    assert ex["D"] is not None
    ms = ft.ModelSet([dict(max=p, max_entropy=pe, beta0=d["beta0"], mu0=d["mu0"], alpha=d["alpha"])])
    s = run(ft, ms, [H], [mu], [kT])
    assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - ex["D"])) < TOL_D
    assert abs(float(s.S.cpu()[0]) - ex["S"]) / 512 < 1e-6
    assert ms.table(0)[0].size == ft.max_nparams(L)


def test_ragged_batch_mixing_families(ft, golden):
    # the Max-SP2 table (small beta') and the printed Eq. mlsp2 table (beta'
    # beyond the Max table's region) in one FP32 solve; the instances start at
    # different layers of the same launches
    d = golden
    ms = ft.ModelSet([dict(theta=tables.PRINTED_B1500, beta0=1500.0, mu0=1.0 / 3.0, alpha=0.842704),
                      dict(max=d["max"], max_entropy=d["max_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                           alpha=d["alpha"])])
    Hs = [wl.chain_1d(300, 4), wl.lattice_3d((8, 8, 8), 2), wl.chain_1d(129, 3)]
    mus, kTs = [0.1, -0.2, 0.0], [0.2, 0.08, 0.3]
    s = run(ft, ms, Hs, mus, kTs)
    rec = s.records()
    assert list(rec["model"]) == [1, 0, 1]
    from oracle import pipeline, rescale
    printed = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
    for b, H in enumerate(Hs):
        if rec["model"][b] == 1:
            ex = maxsp2.method_exact(H, mus[b], kTs[b], d["max"], d["L"], d["beta0"], d["mu0"], d["alpha"],
                                     d["max_entropy"], d["L"])
        else:
            ex = pipeline.method_exact(H, mus[b], kTs[b], [printed])
        assert np.max(np.abs(s.matrix(b).double().cpu().numpy() - ex["D"])) < TOL_D, b
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6


def test_workspace_and_refused_modes(ft, golden):
    d = golden
    ms = max_set(ft, d)
    Hs = [wl.chain_1d(256, 2)]
    host, _, _ = ft._instances([256], [0.0], [0.2])
    a, b = C.c_size_t(), C.c_size_t()
    assert ft.lib().ftsp2_workspace_size(host, 1, ft.FP32, 3, C.byref(a)) == 0
    assert ft.lib().ftsp2_workspace_size_set(host, 1, ms.handle, ft.FP32, 3, C.byref(b)) == 0
    # L + 1 state planes per chain instead of 2
    assert b.value - a.value >= 2 * (d["L"] - 1) * 256 * 256 * 4
    # a workspace sized without the set is refused before any launch
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    raw = np.frombuffer(bytes(host), dtype=np.uint8).copy()
    d_inst = torch.from_numpy(raw).cuda()
    D = torch.full((256 * 256,), float("nan"), dtype=torch.float32, device="cuda")
    rec = torch.zeros(64, dtype=torch.uint8, device="cuda")
    ws = torch.empty(a.value + 1024, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 1023) // 1024 * 1024
    st = ft.lib().ftsp2_density(C.c_void_p(Hd.data_ptr()), host, C.c_void_p(d_inst.data_ptr()), 1, ms.handle,
                                ft.FP32, ft.SYNC, C.c_void_p(D.data_ptr()), None, C.c_void_p(rec.data_ptr()),
                                C.c_void_p(wp), a.value, None)
    assert st == ft._lib.E_WORKSPACE
    assert torch.isnan(D).all()
    for mode in ("fp16x2", "bf16x3", "tf32x3"):
        with pytest.raises(ft.Ftsp2Error) as e:
            run(ft, ms, Hs, [0.0], [0.2], mode=mode, want=1)
        assert e.value.code == ft._lib.E_UNSUPPORTED


def _bounded_max_table(rng, L):
    # u_i = 0.3 + 0.5 x_i + small weights on the earlier layers: x stays in
    # [0, 1] for x_0 in [0, 1], so every layer is well conditioned
    delta, gamma, theta = np.full(L, 0.3), rng.uniform(-0.3, 0.3, L + 1), []
    for i in range(L):
        th = rng.uniform(-0.05, 0.05, i + 1)
        th[i] = 0.5
        theta.append(th)
    return maxsp2.flat(delta, gamma, theta, 0.1)


@pytest.mark.parametrize("L", [1, 2, 20])
def test_depth_limits_and_tiny_orders(ft, L):
    # one layer (the first layer is the last), two, and the largest table
    # (20 layers, 21 state planes per chain); orders 1, 17 and 130 (ragged,
    # below one tile, across a tile edge)
    rng = np.random.default_rng(L)
    p, pe = _bounded_max_table(rng, L), _bounded_max_table(rng, L)
    d = dict(beta0=100.0, mu0=1.0 / 3.0, alpha=0.842704)
    ms = ft.ModelSet([dict(max=p, max_entropy=pe, **d)])
    Hs = [np.array([[0.3]]), wl.chain_1d(17, 2), wl.chain_1d(130, 8)]
    mus, kTs = [0.0, 0.1, -0.1], [0.5, 0.3, 0.25]
    s = run(ft, ms, Hs, mus, kTs)
    for b, H in enumerate(Hs):
        ex = maxsp2.method_exact(H, mus[b], kTs[b], p, L, d["beta0"], d["mu0"], d["alpha"], pe, L)
        if ex["D"] is None:
            assert s.records()[b]["status"] != 0
            continue
        assert s.records()[b]["status"] == 0
        assert np.max(np.abs(s.matrix(b).double().cpu().numpy() - ex["D"])) < TOL_D, (L, b)
        assert abs(float(s.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6
    # the workspace holds L + 1 planes per chain: L = 20 is the limit
    if L == 20:
        with pytest.raises(Exception):
            ft.ModelSet([dict(max=np.zeros(ft.max_nparams(21)), **d)])


@pytest.mark.parametrize("want", [1, 2])
def test_density_only_and_entropy_only(ft, golden, want):
    # one chain per call: the Fermi chain alone (D, traces) or the entropy
    # chain alone (S), each against the oracle and against the two-chain call
    d = golden
    Hs = [wl.lattice_3d((8, 8, 8), 2), wl.chain_1d(200, 7)]
    mus, kTs = [-0.2, 0.1], [0.3, 0.2]
    ms = max_set(ft, d)
    both = run(ft, ms, Hs, mus, kTs, want=3)
    one = run(ft, ms, Hs, mus, kTs, want=want)
    for b, H in enumerate(Hs):
        ex = maxsp2.method_exact(H, mus[b], kTs[b], d["max"], d["L"], d["beta0"], d["mu0"], d["alpha"],
                                 d["max_entropy"], d["L"])
        if want == 1:
            D = one.matrix(b)
            assert torch.equal(D, both.matrix(b))
            assert np.max(np.abs(D.double().cpu().numpy() - ex["D"])) < TOL_D
        else:
            assert float(one.S.cpu()[b]) == float(both.S.cpu()[b])
            assert abs(float(one.S.cpu()[b]) - ex["S"]) / H.shape[0] < 1e-6


def test_ragged_batch_with_lanczos_bounds(ft, golden):
    # Lanczos-tightened bounds and the fewest-layers policy over a set of the
    # printed Eq. mlsp2 table and the Max-SP2 table, FP32 mode, against the
    # oracle's method-exact result with the same bounds and policy
    d = golden
    from oracle import mlsp2, rescale
    ms = ft.ModelSet([dict(theta=tables.PRINTED_B1500, beta0=1500.0, mu0=1.0 / 3.0, alpha=0.842704),
                      dict(max=d["max"], max_entropy=d["max_entropy"], beta0=d["beta0"], mu0=d["mu0"],
                           alpha=d["alpha"])])
    metas = [rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, 0.842704, name="printed"),
             rescale.Table(tuple((0.0, 0.0, 0.0, 0.0) for _ in range(d["L"])), d["beta0"], d["mu0"], d["alpha"])]
    Hs = [wl.chain_1d(150, 1), wl.lattice_3d((8, 8, 8), 3), wl.chain_1d(260, 5)]
    mus, kTs = [0.0, 0.1, -0.1], [0.15, 0.1, 0.05]
    s = run(ft, ms, Hs, mus, kTs, flags=ft.LANCZOS | ft.MIN_LAYERS)
    rec = s.records()
    used = set()
    for b, H in enumerate(Hs):
        _, r = rescale.rescale(H, mus[b], kTs[b], metas, lanczos=True, min_layers=True)
        assert r.valid and rec["status"][b] == 0 and int(rec["model"][b]) == r.model, b
        used.add(r.model)
        eps, V = np.linalg.eigh(H)
        x0 = rescale.x0_of_eigenvalue(eps, mus[b], kTs[b], r, metas[r.model])
        if r.model == 1:
            f = maxsp2.max_scalar(x0, d["max"], d["L"])
            sv = maxsp2.forward(d["max_entropy"], d["L"], x0, "entropy", d["alpha"], d["mu0"])
        else:
            th = np.array(tables.PRINTED_B1500)
            f = mlsp2.mlsp2_scalar(x0, th)
            sv = mlsp2.entropy_scalar(x0, th, 0.842704, 1.0 / 3.0)     # the theta_fermi entropy
        if r.flip:
            f = 1.0 - f
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - (V * f) @ V.T)) < TOL_D, b
        assert abs(float(s.S.cpu()[b]) - float(np.sum(sv))) / H.shape[0] < 1e-6, b
    assert used == {0, 1}
