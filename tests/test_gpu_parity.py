"""GPU parity of the hot path (a1)-(a6) against the CPU oracle, through the C ABI.

Every case compares the library's D (FP32) and S with
  * D_rec / S_rec: the oracle's FP64 scalar recursion on the eigenvalues of H
    (isolates the implementation's rounding), and
  * D_ref / S_ref: the Fermi function and entropy by eigendecomposition
    (total error = model fit error + rounding).
The tolerance is the 1e-6 bound of the FP32-class paths, for every mode; the
few cases with a larger bound say why next to it.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import fermi, mlsp2, pipeline, rescale, sp2, tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRINTED = rescale.Table(tables.PRINTED_B1500, 1500.0, 1.0 / 3.0, name="printed")
MODES = ["fp32", "tf32x3", "bf16x3", "fp16x2"]
# max |D - D_rec| and |S - S_rec| / n allowed for the printed beta0 = 1500
# table: 1e-6.  A layer's rounding is amplified by up to the slope beta0 / 4 of
# the table; the accumulation-chunk setting of each mode (64-element chunks for
# the last 12 FP16X2 layers, for every BF16X3 and TF32X3 layer) keeps the split
# modes inside the bound (measured 5e-7 to 9e-7 at n = 1024 .. 4096).
TOL_D = {"fp32": 1e-6, "tf32x3": 1e-6, "bf16x3": 1e-6, "fp16x2": 1e-6}
TOL_S = 1e-6          # |S - S_rec| / n


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2605_08523_gb300 as ft
    return ft


@pytest.fixture(scope="module")
def printed_set(ft):
    return ft.ModelSet()


def solve(ft, ms, Hs, mus, kTs, mode, want=3, flags=0):
    s = ft.Solver([H.shape[0] for H in Hs], mus, kTs, ms, mode=mode, want=want, flags=flags)
    flat, _ = wl.pack_batch(Hs)
    s.run(torch.from_numpy(flat).cuda(), sync=True)
    torch.cuda.synchronize()
    return s


def check_instance(s, b, H, mu, kT, tabs, mode, tolD=None, tolS=None, clamp=False):
    ex = pipeline.method_exact(H, mu, kT, tabs, clamp=clamp)
    rec = s.records()[b]
    assert rec["status"] == 0
    assert rec["model"] == ex["rec"].model
    assert bool(rec["flip"]) == ex["rec"].flip
    n = H.shape[0]
    tolD = TOL_D[mode] if tolD is None else tolD
    tolS = TOL_S if tolS is None else tolS
    if s.want & 1:
        D = s.matrix(b).double().cpu().numpy()
        assert np.max(np.abs(D - D.T)) == 0.0                  # written symmetric
        err = np.max(np.abs(D - ex["D"]))
        assert err < tolD, (mode, n, err)
        tr = s.trace.cpu().numpy()[b]
        assert abs(tr[0] - ex["trD"]) < max(1e-4, 50 * tolD * math.sqrt(n))
        assert abs(tr[0] - np.trace(D)) < 1e-3
        assert abs(tr[1] - np.sum(D * D)) < 1e-3 * max(1.0, tr[1])
    if s.want & 2:
        S = float(s.S.cpu()[b])
        assert abs(S - ex["S"]) / n < tolS, (mode, n, S, ex["S"])
    return ex


@pytest.mark.parametrize("mode", MODES)
def test_chain256_printed_table(ft, printed_set, mode):
    # the chain workload: open 1D chain n = 256, mu = 0, kT = 0.1 eV.
    H = wl.chain_1d(256, 0)
    s = solve(ft, printed_set, [H], [0.0], [0.1], mode)
    check_instance(s, 0, H, 0.0, 0.1, [PRINTED], mode)
    Dref, Sref, _, _ = fermi.eig_reference(H, 0.0, 0.1)
    assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - Dref)) < TOL_D[mode] + 5e-8


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 127, 128, 129, 255, 257, 300, 383, 513])
def test_ragged_sizes_fp16x2(ft, printed_set, n):
    # sizes around every tile edge (128-row and 256-column tiles) and the tiny cases
    H = wl.chain_1d(n, 10 + n) if n > 1 else np.array([[0.25]])
    mu = 0.1
    s = solve(ft, printed_set, [H], [mu], [0.1], "fp16x2")
    check_instance(s, 0, H, mu, 0.1, [PRINTED], "fp16x2")


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "fp32"])
@pytest.mark.parametrize("n", [129, 300])
def test_ragged_sizes_other_modes(ft, printed_set, mode, n):
    H = wl.chain_1d(n, 20 + n)
    s = solve(ft, printed_set, [H], [-0.2], [0.15], mode)
    check_instance(s, 0, H, -0.2, 0.15, [PRINTED], mode)


@pytest.mark.parametrize("mode", MODES)
def test_lattice_1024(ft, printed_set, mode):
    # the lattice workload at its smallest size: 8 x 8 x 16, mu at half filling.
    H = wl.lattice_3d((8, 8, 16), 0)
    kT = 0.1
    mu = fermi.mu_at_filling(np.linalg.eigvalsh(H), kT, 512)
    s = solve(ft, printed_set, [H], [mu], [kT], mode)
    check_instance(s, 0, H, mu, kT, [PRINTED], mode)


def test_flip_branch(ft, printed_set):
    # mu near the top of the spectrum -> mu' < 1/2 without flip; near the
    # bottom -> flip (Eq. flip).  Both branches against the oracle.
    H = wl.chain_1d(200, 5)
    lo, hi = rescale.gershgorin(H)
    for mu in (lo + 0.3 * (hi - lo), lo + 0.7 * (hi - lo)):
        s = solve(ft, printed_set, [H], [mu], [0.3], "fp16x2")
        ex = check_instance(s, 0, H, mu, 0.3, [PRINTED], "fp16x2")
    assert True


def test_batch_statuses_and_isolation(ft, printed_set):
    # A ragged batch where one instance is outside every region of validity
    # (kT far too low) and one holds a NaN: those report their status, the
    # others are unaffected.
    Hs = [wl.chain_1d(n, 30 + n) for n in (100, 64, 170, 90)]
    Hs[3] = Hs[3].copy()
    Hs[3][5, 7] = np.nan
    mus, kTs = [0.0, 0.1, -0.1, 0.0], [0.1, 1e-4, 0.2, 0.1]
    s = solve(ft, printed_set, Hs, mus, kTs, "fp16x2")
    rec = s.records()
    assert rec["status"][1] == -4 and rec["status"][3] == -5
    assert rec["model"][1] == -1
    for b in (0, 2):
        check_instance(s, b, Hs[b], mus[b], kTs[b], [PRINTED], "fp16x2")
    assert np.isnan(s.trace.cpu().numpy()[1, 0]) and np.isnan(float(s.S.cpu()[3]))


def test_clamp_flag(ft, printed_set):
    H = wl.chain_1d(150, 3)
    mu, kT = 0.05, 0.004
    s = solve(ft, printed_set, [H], [mu], [kT], "fp16x2", flags=ft.CLAMP)
    ex = pipeline.method_exact(H, mu, kT, [PRINTED], clamp=True)
    rec = s.records()[0]
    assert rec["status"] == 0 and rec["valid"] == 0
    assert abs(rec["beta_p"] - ex["rec"].beta_p) < 1e-9 * ex["rec"].beta_p
    D = s.matrix(0).double().cpu().numpy()
    # clamped beta' sits on the edge of the region of validity, where the
    # state spans all of [0, 1] and the rounding amplification is largest
    assert np.max(np.abs(D - ex["D"])) < 2.5e-6


def test_degenerate_spectrum(ft, printed_set):
    H = 0.4 * np.eye(40)
    s = solve(ft, printed_set, [H], [0.38], [0.05], "fp16x2")
    D = s.matrix(0).double().cpu().numpy()
    f = fermi.fermi(np.array([0.4]), 0.38, 0.05)[0]
    assert np.max(np.abs(D - f * np.eye(40))) < 1e-6
    assert s.records()[0]["status"] == 0


def test_entropy_only_and_density_only(ft, printed_set):
    H = wl.chain_1d(190, 9)
    s2 = solve(ft, printed_set, [H], [0.2], [0.12], "fp16x2", want=2)
    s1 = solve(ft, printed_set, [H], [0.2], [0.12], "fp16x2", want=1)
    s3 = solve(ft, printed_set, [H], [0.2], [0.12], "fp16x2", want=3)
    check_instance(s2, 0, H, 0.2, 0.12, [PRINTED], "fp16x2")
    check_instance(s1, 0, H, 0.2, 0.12, [PRINTED], "fp16x2")
    # the fused two-chain launch computes exactly what the single-chain ones do
    assert torch.equal(s1.D, s3.D)
    assert float(s2.S[0]) == float(s3.S[0])


@pytest.mark.parametrize("flags", ["REFINE1", "REFINE2"])
def test_refinement_layers(ft, printed_set, flags):
    H = wl.chain_1d(260, 4)
    s = solve(ft, printed_set, [H], [0.1], [0.1], "fp16x2", flags=getattr(ft, flags))
    check_instance(s, 0, H, 0.1, 0.1, [PRINTED], "fp16x2")


@pytest.mark.parametrize("mode", ["fp16x2", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("refine", ["REFINE1", "REFINE2"])
def test_refinement_layers_on_tensor_cores(ft, printed_set, mode, refine):
    # FTSP2_REFINE_TC: the refinement layers run as BF16X3 tensor-core layers;
    # a ragged pair of instances (different start layers) and a lattice
    Hs = [wl.chain_1d(260, 4), wl.lattice_3d((8, 8, 8), 6)]
    mus, kTs = [0.1, 0.0], [0.1, 0.3]
    s = solve(ft, printed_set, Hs, mus, kTs, mode, flags=getattr(ft, refine) | ft.REFINE_TC)
    for b, H in enumerate(Hs):
        check_instance(s, b, H, mus[b], kTs[b], [PRINTED], mode)


def test_deterministic(ft, printed_set):
    H = wl.chain_1d(384, 12)
    a = solve(ft, printed_set, [H], [0.0], [0.1], "fp16x2")
    b = solve(ft, printed_set, [H], [0.0], [0.1], "fp16x2")
    assert torch.equal(a.D, b.D) and torch.equal(a.S, b.S) and torch.equal(a.trace, b.trace)


def test_rescale_records(ft, printed_set):
    Hs = [wl.chain_1d(n, n) for n in (50, 80, 33)]
    mus, kTs = [0.0, 1.5, -0.7], [0.1, 0.2, 0.05]
    flat, _ = wl.pack_batch(Hs)
    rec = ft.ftsp2_rescale(torch.from_numpy(flat).cuda(), [50, 80, 33], mus, kTs, printed_set)
    for b, H in enumerate(Hs):
        _, r = rescale.rescale(H, mus[b], kTs[b], [PRINTED])
        lo, hi = rescale.gershgorin(H)
        assert abs(rec["e_min"][b] - lo) < 1e-12 * max(1, abs(lo))
        assert abs(rec["e_max"][b] - hi) < 1e-12 * max(1, abs(hi))
        assert bool(rec["flip"][b]) == r.flip and rec["model"][b] == r.model
        assert abs(rec["mu_p"][b] - r.mu_p) < 1e-12 and abs(rec["beta_p"][b] - r.beta_p) < 1e-9 * r.beta_p


def test_model_set_selection(ft):
    # Two tables: the printed one (beta0 = 1500) and a 20-layer SP2-mu table
    # at mu0 = 1/3 given beta0 = 4 x its slope at mu0 (fixed coefficients,
    # the chain workload's "plain recursion").  Selection takes the smallest valid beta0;
    # D is compared with the oracle's method-exact result for the chosen table.
    th_sp2 = sp2.sp2_table(1.0 / 3.0, 20)
    b0 = 4.0 * sp2.slope_at(th_sp2, 1.0 / 3.0)
    SP2 = rescale.Table(th_sp2, b0, 1.0 / 3.0, name="sp2")
    ms = ft.ModelSet([dict(theta=tables.PRINTED_B1500, beta0=1500.0, mu0=1 / 3),
                      dict(theta=th_sp2, beta0=b0, mu0=1 / 3)])
    H = wl.chain_1d(256, 0)
    for kT in (1.0, 0.1):
        s = solve(ft, ms, [H], [0.0], [kT], "fp16x2")
        ex = check_instance(s, 0, H, 0.0, kT, [PRINTED, SP2], "fp16x2", tolD=5e-6, tolS=5e-5)
    assert rescale.select_model([PRINTED, SP2], 0.5, 50.0) == 1


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
def test_lattice_n4096_within_the_1e6_bound(ft, printed_set, mode):
    # The bench workload at full size (16 x 16 x 16 lattice, kT = 0.1, mu at
    # half filling): every element of D within 1e-6 of the eigendecomposition
    # reference, traces consistent, S within the model's own error.
    H = wl.lattice_3d((16, 16, 16), 0)
    n, kT = 4096, 0.1
    Dref, Sref, trref, eps = fermi.eig_reference(H, 0.0, kT)
    mu = fermi.mu_at_filling(eps, kT, n / 2)
    Dref, Sref, trref, _ = fermi.eig_reference(H, mu, kT)
    s = solve(ft, printed_set, [H], [mu], [kT], mode)
    assert s.records()[0]["status"] == 0
    D = s.matrix(0).double().cpu().numpy()
    assert np.max(np.abs(D - Dref)) <= 1e-6
    tr = s.trace.cpu().numpy()[0]
    assert abs(tr[0] - trref) < 1e-3
    # theta_fermi + alpha ansatz: S carries the ansatz's own error (Table entropy row theta_fermi)
    assert abs(float(s.S[0]) - Sref) / n < 5e-6


def _json_set(ft, *names):
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return ft.ModelSet.from_json([os.path.join(root, "paper_2605_08523_gb300", "tables", nm + ".json") for nm in names])


def test_lattice_n4096_entropy_with_trained_table(ft):
    # printed Fermi table + the entropy table trained for it: S within 1e-6
    # per state of the eigendecomposition entropy, D unchanged.
    ms = _json_set(ft, "entropy_b1500_L26")
    H = wl.lattice_3d((16, 16, 16), 0)
    n, kT = 4096, 0.1
    eps = np.linalg.eigvalsh(H)
    mu = fermi.mu_at_filling(eps, kT, n / 2)
    Dref, Sref, trref, _ = fermi.eig_reference(H, mu, kT)
    s = solve(ft, ms, [H], [mu], [kT], "fp16x2")
    assert s.records()[0]["status"] == 0
    assert np.max(np.abs(s.matrix(0).double().cpu().numpy() - Dref)) <= 1e-6
    assert abs(float(s.S[0]) - Sref) / n <= 1e-6


def test_trained_table_applied_to_lattice_n4096_bf16x3(ft):
    # A table trained on the GPU at beta0 = 200, mu0 = 1/3, 32 layers, applied
    # to the n = 4096 lattice in 3xBF16 at kT = 0.5 (beta' ~ 122 <= 2/3 beta0).
    ms = _json_set(ft, "b200_L32")
    H = wl.lattice_3d((16, 16, 16), 0)
    n, kT = 4096, 0.5
    eps = np.linalg.eigvalsh(H)
    mu = fermi.mu_at_filling(eps, kT, n / 2)
    Dref, Sref, _, _ = fermi.eig_reference(H, mu, kT)
    s = solve(ft, ms, [H], [mu], [kT], "bf16x3")
    rec = s.records()[0]
    assert rec["status"] == 0 and rec["model"] == 0
    err = np.max(np.abs(s.matrix(0).double().cpu().numpy() - Dref))
    assert err <= 2e-6          # fit error 6e-7 of the table plus rounding
    assert abs(float(s.S[0]) - Sref) / n <= 2e-6
