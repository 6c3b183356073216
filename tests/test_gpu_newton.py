"""The chemical potential for prescribed electron counts on the GPU
(ftsp2_density_mu) against the oracle's Newton-Raphson solve (Sec. III A 4)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fermi, newton, pipeline, rescale, tables

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


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3", "fp32"])
def test_single_instance_matches_oracle_newton(ft, mode):
    H = wl.lattice_3d((8, 8, 8), 1)
    n, kT = H.shape[0], 0.1
    eps = np.linalg.eigvalsh(H)
    n_occ = 0.5 * n
    mu_exact = fermi.mu_at_filling(eps, kT, n_occ)
    mu0 = mu_exact + 2.5 * kT
    iters, tol = 5, 1e-4
    s = ft.Solver([n], [mu0], [kT], ft.ModelSet(), mode=mode, want=3)
    steps = s.run_mu(torch.from_numpy(H.ravel().copy()).cuda(), [n_occ], iterations=iters, tol=tol, sync=True)
    torch.cuda.synchronize()
    mu_gpu = float(s.mus()[0])
    mu_or, hist, r = newton.newton_mu(H, n_occ, mu0, kT, [PRINTED], iterations=iters, tol=tol)
    assert 1 <= int(steps[0]) <= iters
    # both reach the root of Tr D_rec(mu) = N_occ; they differ by the GPU traces' rounding
    assert abs(mu_gpu - mu_or) < 2e-5, (mu_gpu, mu_or, hist)
    tr = s.trace.cpu().numpy()[0]
    assert abs(tr[0] - n_occ) < 1e-3
    # the returned D and S are those of the final mu
    ex = pipeline.method_exact(H, mu_gpu, kT, [PRINTED])
    D = s.matrix(0).double().cpu().numpy()
    assert np.max(np.abs(D - ex["D"])) < 1e-6
    assert abs(float(s.S.cpu()[0]) - ex["S"]) / n < 1e-6
    # and the root agrees with the exact Fermi root within the model error
    assert abs(mu_gpu - mu_exact) < 1e-4


def test_ragged_batch_independent_instances(ft):
    ns = [300, 128, 257, 90]
    Hs = [wl.chain_1d(m, 80 + m) for m in ns]
    kTs = [0.1, 0.2, 0.15, 0.3]
    fills = [0.5, 0.4, 0.6, 0.3]
    n_occ = [f * m for f, m in zip(fills, ns)]
    mus0, roots = [], []
    for H, kT, N in zip(Hs, kTs, n_occ):
        eps = np.linalg.eigvalsh(H)
        r = fermi.mu_at_filling(eps, kT, N)
        roots.append(r)
        mus0.append(r - 1.5 * kT)
    flat, _ = wl.pack_batch(Hs)
    s = ft.Solver(ns, mus0, kTs, ft.ModelSet(), mode="fp16x2", want=1)
    steps = s.run_mu(torch.from_numpy(flat).cuda(), n_occ, iterations=6, tol=1e-4, sync=True)
    torch.cuda.synchronize()
    mus = s.mus()
    tr = s.trace.cpu().numpy()
    for b, H in enumerate(Hs):
        mu_or, _, _ = newton.newton_mu(H, n_occ[b], mus0[b], kTs[b], [PRINTED], iterations=6, tol=1e-4)
        assert abs(mus[b] - mu_or) < 2e-5, (b, mus[b], mu_or)
        assert abs(tr[b, 0] - n_occ[b]) < 1e-3
        assert abs(mus[b] - roots[b]) < 1e-4
        assert int(steps.cpu()[b]) >= 1


def test_zero_iterations_is_a_plain_solve(ft):
    H = wl.chain_1d(200, 9)
    s = ft.Solver([200], [0.05], [0.1], ft.ModelSet(), mode="fp16x2", want=3)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    steps = s.run_mu(Hd, [100.0], iterations=0, sync=True)
    ref = ft.Solver([200], [0.05], [0.1], ft.ModelSet(), mode="fp16x2", want=3)
    ref.run(Hd, sync=True)
    torch.cuda.synchronize()
    assert int(steps.cpu()[0]) == 0 and float(s.mus()[0]) == 0.05
    assert torch.equal(s.D, ref.D) and torch.equal(s.S, ref.S)


def test_bad_arguments_are_refused(ft):
    H = wl.chain_1d(64, 2)
    s = ft.Solver([64], [0.0], [0.1], ft.ModelSet(), mode="fp16x2", want=1)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    with pytest.raises(ft.Ftsp2Error):
        s.run_mu(Hd, [32.0], iterations=-1)
    with pytest.raises(ft.Ftsp2Error):
        s.run_mu(Hd, [32.0], iterations=2, tol=-1.0)
