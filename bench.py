"""Benchmark of the MLSP2 hot path (density matrix + entropy) on GB300.

Workload (the headline configuration): one dense symmetric H, n = 4096, 3D
cubic tight-binding lattice 16 x 16 x 16 with open boundaries, on-site
U(-1, 1) eV, hopping -1 eV, plus symmetrised 0.01 N(0, 1) dense noise;
kT = 0.1 eV, mu at half filling; the paper's 26-layer table (beta0 = 1500,
mu0 = 1/3) for the density and the entropy table trained for it by the
library's GPU trainer; density and entropy chains; FP16x2 split-precision
tensor-core layers with FP32 accumulation.

A step is one pass of the whole hot path (Gershgorin bounds, rescale, both
26-layer recursions, traces, entropy) over the resident input.  Inputs and
the per-step working set (~0.7 GB) are larger than the 129 MB L2, so no
explicit flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the path has no
exchange step); value = solves of all ranks / max wall time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "density-matrix solves/s and TFLOP/s vs plain FP32 recursion at <=1e-6 error"
LN2 = math.log(2.0)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dims", default="16,16,16")
    p.add_argument("--kT", type=float, default=0.1)
    p.add_argument("--mode", default="fp16x2")
    p.add_argument("--no-baselines", action="store_true")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--mu", type=float, default=None,
                   help="skip the GPU eigendecomposition and use this mu (profiling runs)")
    p.add_argument("--shape", default="auto", choices=["auto", "pair", "single"],
                   help="tensor-core tile shape: auto = the library's autotuner (untimed), or forced")
    p.add_argument("--bounds", default="gershgorin", choices=["gershgorin", "lanczos"],
                   help="spectral bounds: Gershgorin (Appendix A) or tightened by Lanczos (FTSP2_LANCZOS)")
    p.add_argument("--policy", default="beta0", choices=["beta0", "layers"],
                   help="model choice: smallest beta0 (default) or fewest layers (FTSP2_MIN_LAYERS)")
    p.add_argument("--refine", type=int, default=0, choices=[0, 1, 2],
                   help="last 0/1/2 layers in FP32 (FTSP2_REFINE1/2); cfg4 defaults to 2")
    p.add_argument("--epilogue", default="auto", choices=["auto", "deferred", "inline"],
                   help="final epilogue of the pair tiles: the library's default, or forced "
                        "(FTSP2_EPI_DEFERRED / FTSP2_EPI_INLINE)")
    p.add_argument("--operands", default="upper", choices=["upper", "full"],
                   help="operand storage of the 16-bit tensor-core layers: upper triangle with transposed "
                        "panel loads (default), or full matrices (FTSP2_FULL_OPERANDS)")
    p.add_argument("--launch", default="auto", choices=["auto", "layer"],
                   help="consecutive main-format layers in one persistent launch when each layer is a few "
                        "waves of tiles (default), or one launch per layer (FTSP2_LAYER_LAUNCHES)")
    p.add_argument("--batch", type=int, default=512,
                   help="cfg2: number of instances (512; smaller batches for profiling captures)")
    p.add_argument("--table", default="printed", choices=["printed", "alt", "skip"],
                   help="cfg1/cfg4 Fermi table: the paper's printed 26-layer table (with the trained entropy "
                        "table), the 26-layer beta0 = 1500 table of the one-term form (Eq. mlsp2_alt), or the "
                        "26-layer beta0 = 1500 Skip-SP2 table, both trained by the library")
    p.add_argument("--refine-tc", action="store_true",
                   help="refinement layers as BF16X3 tensor-core layers (FTSP2_REFINE_TC)")
    p.add_argument("--workload", default="cfg1", choices=["cfg1", "cfg2", "cfg4"],
                   help="cfg1: the headline single n = 4096 matrix; cfg2: the 512-instance ragged batch; "
                        "cfg4: n = 8192 lattice with 5%% long-range couplings, two FP32 refinement layers "
                        "(cfg2 and cfg4 are separate lines, not the headline)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(dims, seed, longrange=False):
    import workloads as wl
    if longrange:
        return wl.lattice_3d(dims, seed, longrange_frac=0.05, longrange_sigma=0.05)
    return wl.lattice_3d(dims, seed)


def fermi_t(t):
    import torch
    return torch.where(t > 0, torch.exp(-t) / (1 + torch.exp(-t)), 1 / (1 + torch.exp(t)))


def entropy_t(t):
    import torch
    a = t.abs()
    e = torch.exp(-a)
    return torch.log1p(e) + a * e / (1 + e)


def eig_reference_gpu(Hd, kT, n):
    """FP64 eigendecomposition baseline on the GPU: eps, V; mu at half filling;
    D_ref = V f V^T, S_ref = sum s(eps)."""
    import torch
    eps, V = torch.linalg.eigh(Hd)
    lo, hi = float(eps[0]) - 1.0, float(eps[-1]) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if float(fermi_t((eps - mid) / kT).sum()) > n / 2:
            hi = mid
        else:
            lo = mid
    mu = 0.5 * (lo + hi)
    f = fermi_t((eps - mu) / kT)
    D = (V * f[None, :]) @ V.T
    S = float(entropy_t((eps - mu) / kT).sum())
    return mu, D, S, eps, V


def method_exact_gpu(eps, V, rec, table, mu):
    """The method's exact result in FP64 (isolates the library's rounding): the
    scalar recursion of the chosen table on the eigenvalues, with the library's
    own rescale decisions (rec: scale, flip), D_rec = V P(x0) V^T and
    S_rec = sum 4 ln2 F (1 - F) over the entropy chain (Eq. entropy expansion)."""
    import torch
    mu0, alpha = table["mu0"], table["alpha"]
    # X0 = mu0 I + scale (mu I - H): on the eigenvalues x0 = mu0 + scale (mu - eps)
    x = mu0 + float(rec["scale"]) * (mu - eps)
    def chain(x0, th):
        A = torch.zeros_like(x0)
        xx = x0.clone()
        for a, b, c, d in th:
            A = A + d * xx
            xx = a * xx * xx + b * xx + c
        return A + xx

    def chain_skip(x0, tb):
        # Skip-SP2, one stored layer and one accumulator: rows (delta, alpha,
        # beta, gamma), output row (A_0, gamma_L)
        A = torch.full_like(x0, tb[-1][0])
        xx = x0.clone()
        for dl, al, be, ga in tb[:-1]:
            u = dl + al * xx + be * A
            A = A + ga * xx
            xx = u * u
        return A + tb[-1][1] * xx

    if table.get("skip") is not None:
        fermi_f = lambda x0: chain_skip(x0, table["skip"])
        ent_f = lambda x0: chain_skip(x0, table.get("skip_entropy") or table["skip"])
    else:
        fermi_f = lambda x0: chain(x0, table["theta"])
        ent_f = lambda x0: chain(x0, table.get("theta_entropy") or table["theta"])
    P = fermi_f(x)
    if int(rec["flip"]):
        P = 1.0 - P
    Drec = (V * P[None, :]) @ V.T
    F = ent_f(alpha * (x - mu0) + mu0)
    Srec = float((4.0 * LN2 * F * (1.0 - F)).sum())
    return Drec, Srec


def probe_dtype_peaks():
    """Dense-GEMM rates of the dtypes the split modes use (torch.matmul, 8192^3,
    best of 3 after a warm-up, TF32 through allow_tf32), for the hardware
    fractions of FP16X2 and TF32X3: their peak is the measured sustained BF16
    figure times the measured ratio to BF16."""
    import torch
    n = 8192
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16), ("tf32", torch.float32)):
        torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
        a = torch.randn(n, n, device="cuda").to(dt)
        b = torch.randn(n, n, device="cuda").to(dt)
        torch.matmul(a, b)
        t = min(cuda_time(lambda: torch.matmul(a, b), 1) for _ in range(3))
        out[name] = 2.0 * n ** 3 / t / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    return out


def plain_fp32_recursion(Hd, mu, kT, theta, beta0, mu0, alpha, emin, emax):
    """Baseline (i): the plain FP32 recursion of Alg. 2 with torch.matmul
    (TF32 disabled): X and Y chains with the chosen table's Fermi weights."""
    import torch
    n = Hd.shape[0]
    W = emax - emin
    beta = 1.0 / kT
    I = torch.eye(n, dtype=torch.float32, device=Hd.device)
    Hp = (emax * I.double() - Hd) / W
    mup = (emax - mu) / W
    betap = W * beta
    flip = mup > 0.5
    if flip:
        Hp = I.double() - Hp
        mup = 1 - mup
    X = ((betap / beta0) * (Hp - mup * I.double()) + mu0 * I.double()).float()
    Y = alpha * X + (1 - alpha) * mu0 * I
    AD = torch.zeros_like(X)
    AS = torch.zeros_like(X)
    for a, b, c, d in theta:
        AD += d * X
        X = a * (X @ X) + b * X + c * I
        AS += d * Y
        Y = a * (Y @ Y) + b * Y + c * I
    D = AD + X
    if flip:
        D = I - D
    F = AS + Y
    S = 4 * LN2 * (float(torch.trace(F.double())) - float((F.double() ** 2).sum()))
    return D, S


# (mode, n, kernel_sha(): code hash of the layer kernel) -> dram read + write bytes
# of one layer launch (both chains), from the ncu capture summarised in
# profiles/layer_tc_fp16x2_n4096.md
MEASURED_TRAFFIC = {("fp16x2", 4096, "5a532e9ee5962246"): 420.6208e6 + 233.582592e6,
                    ("fp16x2", 4096, "f28e2970fe6099cb"): 422.81472e6 + 233.330176e6,
                    ("fp16x2", 4096, "f2da72eea28cec7d"): 341.659136e6 + 217.101312e6,
                    ("fp16x2", 4096, "35cc88bb61af8eea"): 344.602112e6 + 217.907712e6,
                    ("fp16x2", 4096, "ab8a7663926c8945"): 343.843328e6 + 218.012672e6,
                    ("fp16x2", 4096, "ced6ca48c1eace3f"): 342.698752e6 + 217.683968e6}


def _code_only(src: str) -> str:
    """C/C++ source without comments, blank lines and trailing blanks (string
    and character literals kept), so that comment edits keep the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_sha():
    """sha256[:16] of the layer kernel's code (k_layer_tc.cu, epilogue.cuh,
    ftsp2_internal.h without comments): the key of MEASURED_TRAFFIC."""
    import hashlib
    h = hashlib.sha256()
    for f in ("k_layer_tc.cu", "epilogue.cuh", "ftsp2_internal.h"):
        with open(os.path.join(ROOT, "paper_2605_08523_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def aggregate(t_step_local: float, world: int, device=None):
    """Whole-job throughput of independent replicas: every rank processed one
    solve per step, so value = world / (max over ranks of the step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_step_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t)
    return world / tmax, tmax


def cuda_time(fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


def run_reference(args):
    """Reference arm: the CPU oracle (eigendecomposition definition of D and S)
    timed on the host cores, on a bounded sample of the workload."""
    import numpy as np
    from oracle import fermi
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dims = tuple(int(x) for x in args.dims.split(","))
    n = dims[0] * dims[1] * dims[2]
    sdims = (dims[0] // 2, dims[1], dims[2]) if n > 2048 else dims
    ns = sdims[0] * sdims[1] * sdims[2]
    H = make_workload(sdims, args.seed)
    eps = np.linalg.eigvalsh(H)
    mu = fermi.mu_at_filling(eps, args.kT, ns / 2)
    for _ in range(min(args.warmup, 1)):
        fermi.eig_reference(H, mu, args.kT)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        fermi.eig_reference(H, mu, args.kT)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    scale = (ns / n) ** 3
    value = scale / t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1000 / scale,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "cfg1 lattice %dx%dx%d n=%d kT=%g mu=half filling" % (dims + (n, args.kT)),
                       "n": n, "kT": args.kT},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": "oracle.fermi.eig_reference (numpy eigh + V f V^T + S) on the "
                                       "%dx%dx%d lattice (n=%d) of the same family, scaled to n=%d by n^3"
                                       % (sdims + (ns, n))},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(H, mu, kT, n):
    """The oracle (eigendecomposition definition) timed once on the host cores."""
    from oracle import fermi
    t0 = time.perf_counter()
    fermi.eig_reference(H, mu, kT)
    t = time.perf_counter() - t0
    return {"value": 1.0 / t, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one oracle.fermi.eig_reference solve (numpy eigh + V f V^T + S) of the full n=%d H "
                      "(%.1f s)" % (n, t)}


def run_cfg2(args):
    """Ragged batch of --batch (512) rotated-spectrum Hamiltonians (n ~ U{64..768}),
    one grouped launch per layer for all instances and both chains, model set
    of every shipped table (smallest valid beta0 per instance)."""
    import glob
    import numpy as np
    import torch
    import paper_2605_08523_gb300 as ft
    import workloads as wl
    from paper_2605_08523_gb300 import build as ftbuild
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ftbuild.build()
    tdir = os.path.join(ROOT, "paper_2605_08523_gb300", "tables")
    paths = [os.path.join(tdir, "entropy_b1500_L26.json")] + sorted(glob.glob(os.path.join(tdir, "b*_L32.json")))
    paths += sorted(p for p in glob.glob(os.path.join(tdir, "b*.json"))
                    if int(os.path.basename(p)[1:].split("_")[0]) >= 3000)
    ms = ft.ModelSet.from_json(paths)
    batch = wl.ragged_batch(args.batch, args.seed)
    Hs = [b["H"] for b in batch]
    ns = [H.shape[0] for H in Hs]
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    shape_flag = {"auto": 0, "pair": ft.PAIR_TILES, "single": ft.SINGLE_TILES}[args.shape]
    shape_flag |= {"auto": 0, "deferred": ft.EPI_DEFERRED, "inline": ft.EPI_INLINE}[args.epilogue]
    shape_flag |= ft.FULL_OPERANDS if args.operands == "full" else 0
    shape_flag |= ft.LAYER_LAUNCHES if args.launch == "layer" else 0
    if args.bounds == "lanczos":
        shape_flag |= ft.LANCZOS
    if args.policy == "layers":
        shape_flag |= ft.MIN_LAYERS
    solver = ft.Solver(ns, [b["mu"] for b in batch], [b["kT"] for b in batch], ms, mode=args.mode, want=3,
                       flags=shape_flag)
    if args.shape == "auto":
        shape, ms_single, ms_pair = solver.autotune(Hd, reps=1)
    else:
        shape, ms_single, ms_pair = solver.tile_shape()[0], None, None
    for _ in range(args.warmup):
        solver.run(Hd)
    torch.cuda.synchronize()
    rec = solver.records()
    layers = rec["layers"]
    valid = rec["status"] == 0
    steps = max(3, args.steps // 10)
    t = cuda_time(lambda: solver.run(Hd), steps)
    alg = float(np.sum((np.array(ns, dtype=np.float64) ** 3 * 2 * layers)[valid]))
    # accuracy on a sample of 32 instances (FP64 eigendecomposition on the GPU)
    errD, errS = 0.0, 0.0
    for b in range(0, len(ns), max(1, len(ns) // 32)):
        n_b = ns[b]
        Hb = torch.from_numpy(Hs[b]).cuda()
        eps, V = torch.linalg.eigh(Hb)
        tt = (eps - batch[b]["mu"]) / batch[b]["kT"]
        Dref = (V * fermi_t(tt)[None, :]) @ V.T
        errD = max(errD, float((solver.matrix(b).double() - Dref).abs().max()))
        errS = max(errS, abs(float(solver.S[b]) - float(entropy_t(tt).sum())) / n_b)
    line = {"metric": "ragged-batch solves/s (instances/s, density + entropy)", "value": int(valid.sum()) / t,
            "unit": "solves/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "dtype": args.mode, "data": "synthetic",
            "config": {"workload": "cfg2 ragged batch %d x n~U{64..768}, eigenvalues U(-10,10), kT~U(0.02,0.5), "
                                   "mu~U(-5,5)" % args.batch, "valid_instances": int(valid.sum()),
                       "sum_n3": float(np.sum(np.array(ns, dtype=np.float64) ** 3)),
                       "models_used": {int(m): int(np.sum(rec["model"] == m)) for m in np.unique(rec["model"])},
                       "bounds": args.bounds, "policy": args.policy, "global_layers": int(rec["layers"].max()),
                       "tile_shape": {1: "256x256 CTA pairs", 0: "128x128 single CTAs", -1: "none"}[shape],
                   "epilogue": args.epilogue,
                       "autotune_ms": {"single": ms_single, "pair": ms_pair}},
            "tflops_alg": alg / t / 1e12,
            "accuracy_sampled": {"instances": len(range(0, len(ns), max(1, len(ns) // 32))),
                                 "max_abs_D_minus_Dref": errD, "max_abs_S_minus_Sref_per_n": errS}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "cfg2":
        run_cfg2(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2605_08523_gb300 as ft
    from paper_2605_08523_gb300 import build as ftbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0:
        ftbuild.build()
    if world > 1:
        dist.barrier()
    ft.lib()
    cfg4 = args.workload == "cfg4"
    dims = (16, 16, 32) if cfg4 else tuple(int(x) for x in args.dims.split(","))
    n = dims[0] * dims[1] * dims[2]
    kT = args.kT
    H = make_workload(dims, args.seed + rank, longrange=cfg4)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    Hm = Hd.view(n, n)

    # mu at half filling from the FP64 GPU eigendecomposition (baseline ii)
    torch.backends.cuda.matmul.allow_tf32 = False
    if args.mu is None:
        mu, Dref, Sref, eps, V = eig_reference_gpu(Hm, kT, n)
    else:
        mu, Dref, Sref, eps, V = args.mu, None, None, None, None
    # the paper's printed Fermi table with the entropy table the library's
    # trainer fitted for it (theta_entropy)
    tdir = os.path.join(ROOT, "paper_2605_08523_gb300", "tables")
    tabs = [os.path.join(tdir, {"alt": "alt_b1500_L26.json", "skip": "skip_b1500_L26.json"}.get(
        args.table, "entropy_b1500_L26.json"))]
    if cfg4:
        # the long-range couplings widen the Gershgorin interval: beta' needs the
        # 34-layer beta0 = 3000 table
        tabs.append(os.path.join(tdir, "b3000_L34.json"))
    ms = ft.ModelSet.from_json(tabs)
    shape_flag = {"auto": 0, "pair": ft.PAIR_TILES, "single": ft.SINGLE_TILES}[args.shape]
    shape_flag |= {"auto": 0, "deferred": ft.EPI_DEFERRED, "inline": ft.EPI_INLINE}[args.epilogue]
    shape_flag |= ft.FULL_OPERANDS if args.operands == "full" else 0
    shape_flag |= ft.LAYER_LAUNCHES if args.launch == "layer" else 0
    refine = 2 if cfg4 and args.refine == 0 else args.refine
    shape_flag |= {0: 0, 1: ft.REFINE1, 2: ft.REFINE2}[refine]
    if args.refine_tc:
        shape_flag |= ft.REFINE_TC
    if args.bounds == "lanczos":
        shape_flag |= ft.LANCZOS
    solver = ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=3, flags=shape_flag)
    if args.shape == "auto":
        # tile shape: the library's autotuner times both shapes once (untimed)
        shape, ms_single, ms_pair = solver.autotune(Hd, reps=2)
    else:
        shape, ms_single, ms_pair = solver.tile_shape()[0], None, None
    for _ in range(args.warmup):
        solver.run(Hd)
    torch.cuda.synchronize()
    rec = solver.records()[0]
    if rec["status"] != 0:
        raise SystemExit("hot path status %d (%s)" % (rec["status"], ft.status_string(int(rec["status"]))))

    # ---- timed region (device-resident inputs) ----
    L = int(rec["layers"])
    ft.profile_layers(True)
    ft.profile_read()
    launches0 = ft.kernel_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            solver.run(Hd)
        ev1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ft.kernel_launch_count() - launches0
    layer_ms, layer_n = ft.profile_read()
    ft.profile_layers(False)
    value, t_step = aggregate(ev0.elapsed_time(ev1) / 1000.0 / args.steps, world, device="cuda")
    alg_flops = 2 * L * float(n) ** 3          # L symmetric squares (n^3) per chain, 2 chains
    # ---- accuracy of this run's output ----
    D = solver.matrix(0).double()
    S = float(solver.S[0])
    err_D = float((D - Dref).abs().max()) if Dref is not None else None
    err_S = abs(S - Sref) / n if Sref is not None else None
    trD = float(solver.trace[0, 0])
    err_Drec = err_Srec = None
    if Dref is not None:
        # the model set's table (one-term tables as their converted rows)
        Drec, Srec = method_exact_gpu(eps, V, rec, ms.tables[int(rec["model"])], mu)
        err_Drec = float((D - Drec).abs().max())
        err_Srec = abs(S - Srec) / n
        del Drec

    # density only (no entropy chain): solves/s of the same call with want = 1
    solver_d = ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=1, flags=shape_flag)
    solver_d.run(Hd)
    torch.cuda.synchronize()
    t_density = cuda_time(lambda: solver_d.run(Hd), max(3, args.steps // 4))
    del solver_d

    # ---- end to end through the public API with host buffers ----
    # Every step copies its H from pinned host memory and reads D, S and the
    # traces back.  Two solvers alternate so that the copies of one step run on
    # their own streams while the other step computes: H -> device of step i+1
    # and D -> host of step i-1 overlap step i.
    Hh = torch.from_numpy(H.ravel().copy()).pin_memory()
    Dh = [torch.empty(n * n, dtype=torch.float32).pin_memory() for _ in range(2)]
    Sh = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    Th = [torch.empty(2, dtype=torch.float64).pin_memory() for _ in range(2)]
    Hdev = [torch.empty_like(Hd) for _ in range(2)]
    solvers = [solver, ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=3, flags=shape_flag)]
    comp = torch.cuda.current_stream()
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(steps):
        ev_h2d = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_d2h = [torch.cuda.Event() for _ in range(2)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        s_h2d.wait_event(e0)
        for i in range(steps):
            k = i % 2
            if i >= 2:
                s_h2d.wait_event(ev_done[k])        # step i-2 has consumed Hdev[k]
            with torch.cuda.stream(s_h2d):
                Hdev[k].copy_(Hh, non_blocking=True)
                ev_h2d[k].record(s_h2d)
            comp.wait_event(ev_h2d[k])
            if i >= 2:
                comp.wait_event(ev_d2h[k])          # step i-2's outputs are on the host
            solvers[k].run(Hdev[k], stream=comp)
            ev_done[k].record(comp)
            s_d2h.wait_event(ev_done[k])
            with torch.cuda.stream(s_d2h):
                Dh[k].copy_(solvers[k].D, non_blocking=True)
                Sh[k].copy_(solvers[k].S, non_blocking=True)
                Th[k].copy_(solvers[k].trace[0], non_blocking=True)
                ev_d2h[k].record(s_d2h)
        comp.wait_event(ev_d2h[(steps - 1) % 2])
        if steps >= 2:
            comp.wait_event(ev_d2h[(steps - 2) % 2])
        e1.record(comp)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0 / steps

    e2e_run(2)
    assert torch.equal(Dh[0], Dh[1]) and torch.equal(Dh[0], solver.D.cpu()), "end-to-end outputs differ"
    e2e_steps = max(3, args.steps // 2)
    t_e2e = e2e_run(e2e_steps)
    h2d = n * n * 8
    d2h = n * n * 4 + 8 + 16

    # ---- dominant kernel roofline ----
    pk, pk_kind = peaks()
    # time per layer (both chains): the profiler counts the layers of a
    # multi-layer launch, so flops per layer / time per layer is the launch's rate
    layer_avg = layer_ms / max(1, layer_n) / 1000.0
    alg_per_launch = 2 * float(n) ** 3
    achieved = alg_per_launch / layer_avg / 1e12 if layer_avg > 0 else None
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    # hardware tensor flops actually issued per launch: upper-triangle tiles of
    # the chosen shape x split products x 2 chains
    T = 256 if shape == 1 else 128
    nt = math.ceil(n / T)
    tiles = nt * (nt + 1) // 2
    nprod = {"fp16x2": 3, "tf32x3": 3, "bf16x3": 6}.get(args.mode, 1)
    hw_per_launch = 2 * tiles * T * T * n * 2 * nprod
    hw_achieved = hw_per_launch / layer_avg / 1e12 if layer_avg > 0 else None
    # the split modes' own dtypes: fp16 (FP16X2), bf16 (BF16X3), tf32 (TF32X3);
    # their peak is the measured sustained bf16 figure x the dtype's measured
    # (else nominal) rate ratio to bf16
    dt_of_mode = {"fp16x2": "fp16", "bf16x3": "bf16", "tf32x3": "tf32"}.get(args.mode)
    dtype_rates = probe_dtype_peaks() if (not args.no_baselines and dt_of_mode) else None
    if dtype_rates:
        ratio, ratio_kind = dtype_rates[dt_of_mode] / dtype_rates["bf16"], "measured (torch.matmul 8192^3 probe)"
    else:
        ratio, ratio_kind = {"fp16": 1.0, "bf16": 1.0, "tf32": 1.1 / 2.25}.get(dt_of_mode, 1.0), "nominal"
    hw_peak = peak * ratio
    # DRAM bytes per launch from one ncu capture (profiles/layer_tc_fp16x2_n4096.md),
    # valid only while the kernel sources are the ones that were profiled
    ksha = kernel_sha()
    traffic = MEASURED_TRAFFIC.get((args.mode, n, ksha))

    result = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16x2-split/fp32-accum" if args.mode == "fp16x2" else args.mode,
        "data": "synthetic",
        "config": {"workload": ("cfg4 lattice %dx%dx%d with 5%% long-range couplings N(0,0.05) n=%d kT=%g "
                                "mu=half filling, density+entropy, beta0=1500 and 3000 tables" if cfg4 else
                                "cfg1 lattice %dx%dx%d n=%d kT=%g mu=half filling, density+entropy, "
                                + {"alt": "26-layer beta0=1500 table of the one-term form (Eq. mlsp2_alt)",
                                   "skip": "26-layer beta0=1500 Skip-SP2 table (one stored layer, one accumulator)"}
                                .get(args.table, "printed 26-layer table + trained entropy table"))
                                % (dims + (n, kT)),
                   "n": n, "kT": kT, "mu": mu, "layers": L, "mode": args.mode, "chains": 2,
                   "refine_layers_fp32": refine, "refine_on_tensor_cores": bool(args.refine_tc),
                   "model": int(rec["model"]), "bounds": args.bounds,
                   "e_min": float(rec["e_min"]), "e_max": float(rec["e_max"]),
                   "l2": "inputs and working set larger than L2 (no flush)", "parallelism": "replicas",
                   "tile_shape": {1: "256x256 CTA pairs", 0: "128x128 single CTAs", -1: "none"}[shape],
                   "epilogue": args.epilogue, "table": args.table, "operands": args.operands,
                   "launch": args.launch,
                   "autotune_ms": {"single": ms_single, "pair": ms_pair}},
        "tflops_alg": alg_flops / t_step / 1e12 * world,
        "density_only": {"value": world / t_density, "unit": "solves/s", "ms_per_step": t_density * 1e3},
        "accuracy": {"max_abs_D_minus_Dref": err_D, "abs_S_minus_Sref_per_n": err_S,
                     "max_abs_D_minus_Drec": err_Drec, "abs_S_minus_Srec_per_n": err_Srec, "trD": trD,
                     "trD_ref": n / 2, "S": S, "S_ref": Sref},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "layer_tc_kernel<%s>" % args.mode.upper(), "kernel_sha": ksha,
                     "per_layer_alg_flops": alg_per_launch, "avg_layer_ms": layer_avg * 1000,
                     "work_unit": "one layer of both chains (CUDA events around each layer-kernel launch; "
                                  "a multi-layer launch counts its layers)",
                     "peak_kind": "bf16_tflops_sustained (%s)" % pk_kind,
                     "hw_tensor_tflops": hw_achieved, "hw_frac": (hw_achieved / hw_peak) if hw_achieved else None,
                     "hw_peak": hw_peak, "hw_peak_dtype": dt_of_mode, "hw_peak_ratio_to_bf16": ratio,
                     "hw_peak_ratio_kind": ratio_kind, "dtype_probe_tflops": dtype_rates},
        "e2e": {"value": world / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }

    if not args.no_baselines:
        # baseline (i): plain FP32 recursion with torch.matmul, TF32 off
        th_tab, b0_tab, m0_tab, al_tab = ms.table(int(rec["model"]))
        theta = [tuple(r) for r in th_tab]
        emin, emax = float(rec["e_min"]), float(rec["e_max"])
        out = {}

        def fp32_step():
            out["r"] = plain_fp32_recursion(Hm, mu, kT, theta, b0_tab, m0_tab, al_tab, emin, emax)

        fp32_step()
        t32 = cuda_time(fp32_step, 2)
        D32, S32 = out["r"]
        t64 = cuda_time(lambda: eig_reference_gpu(Hm, kT, n), 1)
        result["baselines"] = {
            "plain_fp32_recursion": {"solves_per_s": 1 / t32, "max_abs_D_minus_Dref": float((D32.double() - Dref).abs().max()),
                                     "abs_S_minus_Sref_per_n": abs(S32 - Sref) / n,
                                     "math": "torch.matmul fp32, allow_tf32=False"},
            "fp64_eigh_gpu": {"solves_per_s": 1 / t64, "how": "torch.linalg.eigh float64 + V f V^T + S"},
            "speedup_vs_fp32_recursion": value / world * t32,
            "speedup_vs_fp64_eigh": value / world * t64,
        }
    if rank == 0 and world == 1 and not args.no_baselines:
        result["cpu_baseline"] = cpu_baseline(H, mu, kT, n)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
