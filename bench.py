"""Benchmark of the MLSP2 hot path (density matrix + entropy) on GB300.

Default workload (the largest single-GPU configuration): one dense symmetric H,
n = 8192, open 3D cubic tight-binding lattice 16 x 16 x 32 (on-site U(-1, 1)
eV, hopping -1 eV, symmetrised 0.01 N(0, 1) dense noise) with 5 % of the
off-diagonal pairs given long-range couplings N(0, 0.05) eV; kT = 0.1 eV, mu
at half filling; Gershgorin bounds; model set = the paper's printed 26-layer
table (beta0 = 1500, with the entropy table the library's trainer fitted for
it) and the library-trained 34-layer beta0 = 3000 table, which the Gershgorin
width of this matrix selects; FP16X2 split-precision tensor-core layers with
FP32 accumulation, the last two layers as FP32-class refinement layers
(BF16X3 products on the tensor cores); density and entropy chains.

A step is one pass of the whole hot path (Gershgorin bounds, rescale, both
recursions, traces, entropy) over the resident input.  Inputs and the per-step
working set (several GB) are larger than the 129 MB L2, so no explicit flush is
needed between steps.

Other workloads (--workload): ``lattice`` (one n = 1024 / 2048 / 4096 lattice
without the long-range couplings) and ``ragged`` (512 rotated-spectrum
Hamiltonians, n ~ U{64..768}, one grouped launch per layer for all instances,
timed as CUDA-graph replays; under torchrun the batch is split across ranks in
shares of equal sum n^3).  The default run also measures the ragged batch and
the n = 4096 lattice as secondary results in the same JSON line.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica of a single-matrix
workload (the path has no exchange step); value = solves of all ranks / max
time over ranks.
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
TABLE_DIR = os.path.join(ROOT, "paper_2605_08523_gb300", "tables")


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="longrange", choices=["longrange", "lattice", "ragged", "families"],
                   help="longrange: n = 8192 lattice with 5%% long-range couplings, two refinement layers "
                        "(default); lattice: one lattice of --dims; ragged: the 512-instance ragged batch; "
                        "families: the beta0 = 100 tables of Eq. mlsp2, Max-SP2 and Skip-SP2 (k = K = 2) on "
                        "one lattice of --dims in FP32 mode (use --kT 0.3)")
    p.add_argument("--dims", default="16,16,16", help="lattice workload: lattice dimensions")
    p.add_argument("--kT", type=float, default=0.1)
    p.add_argument("--mode", default="fp16x2")
    p.add_argument("--no-baselines", action="store_true")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the secondary measurements (ragged batch, n = 4096 lattice) of the default run")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--mu", type=float, default=None,
                   help="skip the GPU eigendecomposition and use this mu (profiling runs)")
    p.add_argument("--shape", default="auto", choices=["auto", "pair", "single"],
                   help="tensor-core tile shape: auto = the library's autotuner (untimed), or forced")
    p.add_argument("--bounds", default=None, choices=["gershgorin", "lanczos"],
                   help="spectral bounds: Gershgorin (Appendix A; single-matrix default) or tightened by Lanczos "
                        "(FTSP2_LANCZOS; ragged default)")
    p.add_argument("--policy", default=None, choices=["beta0", "layers"],
                   help="model choice: smallest beta0 (single-matrix default) or fewest layers "
                        "(FTSP2_MIN_LAYERS; ragged default)")
    p.add_argument("--refine", type=int, default=None, choices=[0, 1, 2],
                   help="last 0/1/2 layers as refinement layers (FTSP2_REFINE1/2); longrange defaults to 2")
    p.add_argument("--refine-on", default="tc", choices=["tc", "cuda"],
                   help="refinement layers as BF16X3 tensor-core layers (FTSP2_REFINE_TC, default) or as FP32 "
                        "FMA on the CUDA cores")
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
                   help="ragged: number of instances (512; smaller batches for profiling captures)")
    p.add_argument("--table", default="printed", choices=["printed", "alt", "skip"],
                   help="lattice Fermi table: the paper's printed 26-layer table (with the trained entropy "
                        "table), the 26-layer beta0 = 1500 table of the one-term form (Eq. mlsp2_alt), or the "
                        "26-layer beta0 = 1500 Skip-SP2 table, both trained by the library")
    return p.parse_args(argv)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 100 ms while running."""

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


def single_dims_desc(args):
    """(lattice dimensions, description) of a single-matrix workload."""
    if args.workload == "longrange":
        return (16, 16, 32), ("lattice 16x16x32 (n=8192) with 5%% long-range couplings N(0,0.05), kT=%g, mu at "
                              "half filling, density+entropy" % args.kT)
    dims = tuple(int(x) for x in args.dims.split(","))
    return dims, ("lattice %dx%dx%d (n=%d), kT=%g, mu at half filling, density+entropy"
                  % (dims + (dims[0] * dims[1] * dims[2], args.kT)))


def single_workload(args):
    """(H, dims, description) of a single-matrix workload; rank r uses seed + r."""
    import workloads as wl
    dims, desc = single_dims_desc(args)
    seed = args.seed + int(os.environ.get("RANK", "0"))
    if args.workload == "longrange":
        H = wl.lattice_3d(dims, seed, longrange_frac=0.05, longrange_sigma=0.05)
    else:
        H = wl.lattice_3d(dims, seed)
    return H, dims, desc


def fermi_t(t):
    import torch
    return torch.where(t > 0, torch.exp(-t) / (1 + torch.exp(-t)), 1 / (1 + torch.exp(t)))


def entropy_t(t):
    import torch
    a = t.abs()
    e = torch.exp(-a)
    return torch.log1p(e) + a * e / (1 + e)


def mu_half_filling(eps, kT, n):
    lo, hi = float(eps[0]) - 1.0, float(eps[-1]) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if float(fermi_t((eps - mid) / kT).sum()) > n / 2:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def eig_reference_gpu(Hd, kT, n, mu=None):
    """FP64 eigendecomposition baseline on the GPU: eps, V; mu at half filling
    (unless given); D_ref = V f V^T, S_ref = sum s(eps)."""
    import torch
    eps, V = torch.linalg.eigh(Hd)
    if mu is None:
        mu = mu_half_filling(eps, kT, n)
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

    def chain_max(x0, p):
        # Max-SP2, flat table: blocks (delta_i, gamma_i, theta_{i,0..i}), then (c, gamma_L)
        L = next(l for l in range(1, 64) if l * (l + 5) // 2 + 2 == len(p))
        xs, F, o = [x0], torch.zeros_like(x0), 0
        for i in range(L):
            u = torch.full_like(x0, p[o])
            for j in range(i + 1):
                u = u + p[o + 2 + j] * xs[j]
            F = F + p[o + 1] * xs[i]
            xs.append(u * u)
            o += i + 3
        return F + p[o] + p[o + 1] * xs[L]

    if table.get("max") is not None:
        fermi_f = lambda x0: chain_max(x0, table["max"])
        ent_f = lambda x0: chain_max(x0, table.get("max_entropy") or table["max"])
    elif table.get("skip") is not None:
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


def plain_fp32_recursion(Hd, mu, kT, theta, beta0, mu0, alpha, emin, emax, theta_entropy=None):
    """Baseline (i): the plain FP32 recursion of Alg. 2 with torch.matmul
    (TF32 disabled): X and Y chains with the chosen table's weights."""
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
    del Hp
    AD = torch.zeros_like(X)
    AS = torch.zeros_like(X)
    for a, b, c, d in theta:
        AD += d * X
        X = a * (X @ X) + b * X + c * I
    for a, b, c, d in (theta_entropy if theta_entropy is not None else theta):
        AS += d * Y
        Y = a * (Y @ Y) + b * Y + c * I
    D = AD + X
    if flip:
        D = I - D
    F = AS + Y
    S = 4 * LN2 * (float(torch.trace(F.double())) - float((F.double() ** 2).sum()))
    return D, S


# (mode, n, kernel_sha(): code hash of the layer kernel) -> DRAM read + write
# bytes of one layer launch of both chains, from an ncu capture of that launch
# (dram__bytes_read.sum + dram__bytes_write.sum) at that code hash
# (mode, batch size, kernel_sha()) -> (DRAM read + write bytes, algorithmic
# bytes) of one ragged-batch layer launch with every instance active, from an
# ncu capture of that launch at that code hash
MEASURED_RAGGED_TRAFFIC = {
    # 512-instance ragged batch, global layer 35 of 44: 1.78 GB read + 1.55 GB
    # written in 0.937 ms
    ("fp16x2", 512, "215c1725bf044bed"): (3.33e9, 3.285e9),
}

MEASURED_TRAFFIC = {
    # n = 8192 long-range lattice, FP16X2 main layer (layer_tc_kernel<FP16X2,
    # FP16X2, pair, deferred>): 3.22 GB read + 1.04 GB written per launch
    ("fp16x2", 8192, "215c1725bf044bed"): 4.26e9,
}


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


def aggregate(t_step_local: float, world: int, units_local: float = 1.0, device=None):
    """Whole-job throughput: every rank processed ``units_local`` units per
    step; value = (sum of units over ranks) / (max over ranks of the step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_step_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    tmax = float(t)
    return float(u) / tmax, tmax


def partition_by_work(ns, world):
    """Split instances of orders ns across `world` ranks in shares of nearly
    equal sum n^3 (the layers' work grows with n^3): largest first, each to the
    currently lightest rank.  Returns one sorted index list per rank."""
    order = sorted(range(len(ns)), key=lambda b: (-int(ns[b]) ** 3, b))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(b)
        load[r] += int(ns[b]) ** 3
    return [sorted(p) for p in parts]


def cuda_time(fn, reps, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


# ---------------------------------------------------------------------------
# configurations shared by both arms
# ---------------------------------------------------------------------------
def overlapped_e2e(solvers, Hh, Hdev, outs, steps, comp, s_h2d, s_d2h):
    """End-to-end steps through the public API: every step copies H from
    pinned host memory (Hh) into Hdev[k], runs solvers[k] (k = step % 2) on the
    compute stream and reads its outputs back into pinned host memory
    (outs[k]: list of (host tensor, device tensor)).  The copies of one step
    run on their own streams while the other solver computes: H of step i + 1
    goes up and the outputs of step i - 1 come down during step i.  Returns
    seconds per step (CUDA events on the compute stream, after every copy)."""
    import torch
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
            for host, dev in outs[k]:
                host.copy_(dev, non_blocking=True)
            ev_d2h[k].record(s_d2h)
    comp.wait_event(ev_d2h[(steps - 1) % 2])
    if steps >= 2:
        comp.wait_event(ev_d2h[(steps - 2) % 2])
    e1.record(comp)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / steps


def single_config(args):
    """The workload description both arms report (inputs only, no results)."""
    dims, desc = single_dims_desc(args)
    n = dims[0] * dims[1] * dims[2]
    longrange = args.workload == "longrange"
    refine = refine_layers_of(args)
    return {"workload": desc, "n": n, "kT": args.kT, "mode": args.mode, "chains": 2,
            "bounds": bounds_of(args), "policy": policy_of(args),
            "tables": ("printed 26-layer beta0=1500 (+ trained entropy table)" if (longrange or args.table == "printed")
                       else args.table) + (" and trained 27-layer beta0=2250, 34-layer beta0=3000"
                                           if (longrange or args.kT < 0.1) else ""),
            "refine_layers": refine, "refine_on": args.refine_on if refine else None,
            "l2": "inputs and working set larger than L2 (no flush)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def ragged_config(args):
    return {"workload": "ragged batch of %d rotated-spectrum Hamiltonians, n~U{64..768}, eigenvalues U(-10,10) eV, "
                        "mu~U(-5,5), kT~U(0.02,0.5), density+entropy" % args.batch,
            "instances": args.batch, "mode": args.mode, "chains": 2, "bounds": bounds_of(args),
            "policy": policy_of(args), "tables": "printed, 32-layer sweep, high-beta0 and polished low-beta0 tables",
            "l2": "inputs and working set larger than L2 (no flush)",
            "parallelism": "instances split across ranks by sum n^3" if args.gpus > 1 else "single GPU"}


def bounds_of(args):
    if args.bounds:
        return args.bounds
    return "lanczos" if args.workload == "ragged" else "gershgorin"


def policy_of(args):
    if args.policy:
        return args.policy
    return "layers" if args.workload == "ragged" else "beta0"


def refine_layers_of(args):
    if args.refine is not None:
        return args.refine
    return 2 if args.workload == "longrange" else 0


# polished low-beta0 tables (fewer layers than the printed one where beta'
# is small); with the fewest-layers policy most instances of the ragged
# batch take one of them.  The shallower b200_L19, b400_L22 and b800_L24 fit
# as well but leave instances of the batch above 1e-6 in TF32X3 mode
RAGGED_LOW = ("b100_L18", "b200_L21", "b400_L24")


def ragged_table_paths():
    """Model set of the ragged batch: the printed table (with its trained
    entropy table), the 32-layer sweep tables, the high-beta0 tables and the
    polished low-beta0 tables."""
    import glob
    paths = [os.path.join(TABLE_DIR, "entropy_b1500_L26.json")]
    paths += sorted(glob.glob(os.path.join(TABLE_DIR, "b*_L32.json")))
    paths += sorted(p for p in glob.glob(os.path.join(TABLE_DIR, "b*.json"))
                    if int(os.path.basename(p)[1:].split("_")[0]) >= 3000)
    paths += [os.path.join(TABLE_DIR, nm + ".json") for nm in RAGGED_LOW]
    return paths


def table_paths(args):
    if args.workload == "ragged":
        return ragged_table_paths()
    first = {"alt": "alt_b1500_L26.json", "skip": "skip_b1500_L26.json"}.get(
        args.table if args.workload == "lattice" else "printed", "entropy_b1500_L26.json")
    paths = [os.path.join(TABLE_DIR, first)]
    # the polished 24-layer beta0 = 1000 table serves the lattice with the
    # printed table's weights where beta' is small enough (kT >= 0.1 on the
    # n = 4096 lattice: beta' ~ 620 at mu' ~ 1/2)
    if args.workload == "lattice" and args.table == "printed":
        paths.append(os.path.join(TABLE_DIR, "b1000_L24.json"))
    # the beta0 = 2250 and 3000 tables serve the cases whose Gershgorin width
    # puts beta' beyond the printed table's region (the long-range couplings,
    # and kT = 0.05 on the n = 4096 lattice); the rescale takes the smallest
    # valid beta0
    if args.workload == "longrange" or args.kT < 0.1:
        paths.append(os.path.join(TABLE_DIR, "b2250_L27.json"))
        paths.append(os.path.join(TABLE_DIR, "b3000_L34.json"))
    return paths


def flags_of(args, ft):
    f = {"auto": 0, "pair": ft.PAIR_TILES, "single": ft.SINGLE_TILES}[args.shape]
    f |= {"auto": 0, "deferred": ft.EPI_DEFERRED, "inline": ft.EPI_INLINE}[args.epilogue]
    f |= ft.FULL_OPERANDS if args.operands == "full" else 0
    f |= ft.LAYER_LAUNCHES if args.launch == "layer" else 0
    r = refine_layers_of(args)
    f |= {0: 0, 1: ft.REFINE1, 2: ft.REFINE2}[r]
    if r and args.refine_on == "tc":
        f |= ft.REFINE_TC
    if bounds_of(args) == "lanczos":
        f |= ft.LANCZOS
    if policy_of(args) == "layers":
        f |= ft.MIN_LAYERS
    return f


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def oracle_sample(args):
    """(callable timing one step, full-workload units per step, description):
    a bounded sample of the workload for the oracle on the host cores."""
    import numpy as np
    import workloads as wl
    from oracle import fermi
    if args.workload == "ragged":
        batch = wl.ragged_batch(args.batch, args.seed)
        ns = np.array([b["n"] for b in batch], dtype=np.float64)
        # every 16th instance in order of size: the sample spans the size range
        pick = list(np.argsort(ns)[::16])
        frac = float(np.sum(ns[pick] ** 3) / np.sum(ns ** 3))

        def step():
            for b in pick:
                fermi.eig_reference(batch[b]["H"], batch[b]["mu"], batch[b]["kT"])
        return step, frac * len(batch), ("oracle.fermi.eig_reference (numpy eigh + V f V^T + S) on %d of the %d "
                                         "instances (every 16th by size, %.3f of the batch's sum n^3); value "
                                         "scaled to instances/s of the whole batch by sum n^3" % (len(pick), len(batch), frac))
    if args.workload == "longrange":
        dims = (16, 16, 16)
        H = wl.lattice_3d(dims, args.seed, longrange_frac=0.05, longrange_sigma=0.05)
        n_full = 8192
    else:
        dims = tuple(int(x) for x in args.dims.split(","))
        H = wl.lattice_3d(dims, args.seed)
        n_full = dims[0] * dims[1] * dims[2]
    n = H.shape[0]
    eps = np.linalg.eigvalsh(H)
    mu = fermi.mu_at_filling(eps, args.kT, n / 2)

    def step():
        fermi.eig_reference(H, mu, args.kT)
    frac = (n / n_full) ** 3
    what = ("the full n=%d matrix" % n if n == n_full else
            "the %dx%dx%d member (n=%d) of the same family, %.3f of the n=%d solve's n^3 work; value scaled "
            "to n=%d solves/s by n^3" % (dims + (n, frac, n_full, n_full)))
    return step, frac, "oracle.fermi.eig_reference (numpy eigh + V f V^T + S) on " + what


def run_reference(args):
    """Reference arm: the CPU oracle (eigendecomposition definition of D and S)
    timed on the host cores; each step is the bounded sample of oracle_sample,
    and the value is in units of the full workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    step, units, sample = oracle_sample(args)
    for _ in range(args.warmup):
        step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    t = sum(ts) / len(ts)
    value = units / t
    cores = os.cpu_count()
    cfg = ragged_config(args) if args.workload == "ragged" else single_config(args)
    unit = "instances/s" if args.workload == "ragged" else "solves/s"
    line = {"impl": "reference", "metric": METRIC if args.workload != "ragged" else
            "ragged-batch instances/s (density + entropy) at <=1e-6 error",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1000.0, "units_per_step": units, "higher_is_better": True,
            "scaling": "strong" if args.workload == "ragged" else "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, reps=3):
    """The oracle on the host cores (rank 0, N = 1): the reference arm's
    bounded sample, median of `reps` steps."""
    step, units, sample = oracle_sample(args)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"value": units / t, "unit": "instances/s" if args.workload == "ragged" else "solves/s",
            "cores": os.cpu_count(), "kind": "oracle", "sample": sample + "; median of %d steps (%.1f s each)"
            % (reps, t)}


# ---------------------------------------------------------------------------
# our arm: one matrix per rank
# ---------------------------------------------------------------------------
def hw_flops_per_solve(n, T, L, R, mode, refine_tc, chains=2):
    """(tensor MMA flops a solve issues, tensor-core layers): upper-triangle
    tiles of side T, each T x T x n per product; 3 products per FP16X2 / TF32X3
    layer, 6 per BF16X3 layer; refinement layers on the tensor cores are BF16X3
    (in BF16X3 mode they are ordinary layers), on the CUDA cores they issue no
    MMAs."""
    if mode == "fp32":
        return 0.0, 0
    nt = math.ceil(n / T)
    per_product = 2.0 * (nt * (nt + 1) // 2) * T * T * n * chains
    nprod = {"fp16x2": 3, "tf32x3": 3, "bf16x3": 6}[mode]
    if refine_tc and mode == "bf16x3":
        R = 0
    ref_tc = R if refine_tc else 0
    return per_product * ((L - R) * nprod + ref_tc * 6), (L - R) + ref_tc


def run_single(args, ft, world, rank, local, secondary=False):
    """One single-matrix workload: the timed hot path, its layer roofline,
    accuracy, end-to-end time through the API with host buffers, baselines.
    Returns the result dict (the JSON line of the run, or a secondary entry)."""
    import torch
    import torch.distributed as dist
    H, dims, desc = single_workload(args)
    n = H.shape[0]
    kT = args.kT
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    Hm = Hd.view(n, n)
    torch.backends.cuda.matmul.allow_tf32 = False
    if args.mu is None:
        mu, Dref, Sref, eps, V = eig_reference_gpu(Hm, kT, n)
    else:
        mu, Dref, Sref, eps, V = args.mu, None, None, None, None
    ms = ft.ModelSet.from_json(table_paths(args))
    flags = flags_of(args, ft)
    R = refine_layers_of(args)
    refine_tc = bool(R) and args.refine_on == "tc"
    solver = ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=3, flags=flags)
    if args.shape == "auto":
        # tile shape: the library's autotuner times both shapes (untimed)
        shape, ms_single, ms_pair = solver.autotune(Hd, reps=2)
    else:
        shape, ms_single, ms_pair = solver.tile_shape()[0], None, None
    for _ in range(max(3, args.warmup)):
        solver.run(Hd)
    torch.cuda.synchronize()
    rec = solver.records()[0]
    if rec["status"] != 0:
        raise SystemExit("hot path status %d (%s)" % (rec["status"], ft.status_string(int(rec["status"]))))
    L = int(rec["layers"])

    # ---- timed region (device-resident inputs, no instrumentation) ----
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
    value, t_step = aggregate(ev0.elapsed_time(ev1) / 1000.0 / args.steps, world, 1.0, device="cuda")

    # ---- layer times: a second timed pass of the same steps with CUDA events
    # recorded around every layer-kernel launch on the launching stream ----
    ft.profile_layers(True)
    ft.profile_read()
    for _ in range(args.steps):
        solver.run(Hd)
    torch.cuda.synchronize()
    layer_ms, layer_n = ft.profile_read()
    ft.profile_layers(False)

    # ---- accuracy of this run's output ----
    D = solver.matrix(0).double()
    S = float(solver.S[0])
    err_D = float((D - Dref).abs().max()) if Dref is not None else None
    err_S = abs(S - Sref) / n if Sref is not None else None
    err_Drec = err_Srec = None
    if Dref is not None:
        Drec, Srec = method_exact_gpu(eps, V, rec, ms.tables[int(rec["model"])], mu)
        err_Drec = float((D - Drec).abs().max())
        err_Srec = abs(S - Srec) / n
        del Drec
    del D
    if V is not None:
        del V
    torch.cuda.empty_cache()

    # ---- density only (no entropy chain) ----
    solver_d = ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=1, flags=flags)
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
    solvers = [solver, ft.Solver([n], [mu], [kT], ms, mode=args.mode, want=3, flags=flags)]
    comp = torch.cuda.current_stream()
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(steps):
        outs = [[(Dh[k], solvers[k].D), (Sh[k], solvers[k].S), (Th[k], solvers[k].trace[0])] for k in range(2)]
        return overlapped_e2e(solvers, Hh, Hdev, outs, steps, comp, s_h2d, s_d2h)

    e2e_run(2)
    assert torch.equal(Dh[0], Dh[1]) and torch.equal(Dh[0], solver.D.cpu()), "end-to-end outputs differ"
    t_e2e = e2e_run(max(3, args.steps // 2))
    e2e_value, _ = aggregate(t_e2e, world, 1.0, device="cuda")
    h2d = n * n * 8
    d2h = n * n * 4 + 8 + 16
    del solvers, Hdev
    torch.cuda.empty_cache()

    # ---- dominant kernel roofline: the tensor-core layer kernel ----
    pk, pk_kind = peaks()
    # mean time of one tensor-core layer: the profiled launches cover every
    # tensor-core layer of the steps (a multi-layer launch counts its layers)
    hw_solve, tc_layers = hw_flops_per_solve(n, 256 if shape == 1 else 128, L, R, args.mode, refine_tc)
    layer_avg = layer_ms / max(1, args.steps * tc_layers) / 1000.0
    alg_per_launch = 2 * float(n) ** 3          # one layer of both chains: n^3 per chain
    achieved = alg_per_launch / layer_avg / 1e12 if layer_avg > 0 else None
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    hw_achieved = hw_solve / (layer_avg * max(1, tc_layers)) / 1e12 if layer_avg > 0 else None
    dt_of_mode = {"fp16x2": "fp16", "bf16x3": "bf16", "tf32x3": "tf32"}.get(args.mode)
    dtype_rates = probe_dtype_peaks() if (not args.no_baselines and dt_of_mode and not secondary) else None
    if dtype_rates:
        ratio, ratio_kind = dtype_rates[dt_of_mode] / dtype_rates["bf16"], "measured (torch.matmul 8192^3 probe)"
    else:
        ratio, ratio_kind = {"fp16": 1.0, "bf16": 1.0, "tf32": 1.1 / 2.25}.get(dt_of_mode, 1.0), "nominal"
    hw_peak = peak * ratio
    ksha = kernel_sha()
    traffic = MEASURED_TRAFFIC.get((args.mode, n, ksha))
    alg_flops = 2 * L * float(n) ** 3           # L symmetric squares (n^3) per chain, 2 chains

    result = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16x2-split/fp32-accum" if args.mode == "fp16x2" else args.mode,
        "data": "synthetic", "config": single_config(args),
        "details": {"mu": mu, "layers": L, "model": int(rec["model"]), "e_min": float(rec["e_min"]),
                    "e_max": float(rec["e_max"]), "beta_p": float(rec["beta_p"]),
                    "tile_shape": {1: "256x256 CTA pairs", 0: "128x128 single CTAs", -1: "none"}[shape],
                    "epilogue": args.epilogue, "operands": args.operands, "launch": args.launch,
                    "autotune_ms": {"single": ms_single, "pair": ms_pair}},
        "tflops_alg": alg_flops / t_step / 1e12 * world,
        "density_only": {"value": world / t_density, "unit": "solves/s", "ms_per_step": t_density * 1e3},
        "accuracy": {"max_abs_D_minus_Dref": err_D, "abs_S_minus_Sref_per_n": err_S,
                     "max_abs_D_minus_Drec": err_Drec, "abs_S_minus_Srec_per_n": err_Srec,
                     "trD": float(solver.trace[0, 0]), "trD_ref": n / 2, "S": S, "S_ref": Sref},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "layer_tc_kernel<%s>" % args.mode.upper(), "kernel_sha": ksha,
                     "per_launch_alg_flops": alg_per_launch, "avg_layer_ms": layer_avg * 1000,
                     "work_unit": "one layer of both chains (n^3 flops per chain: the symmetric square); layer "
                                  "times from a second pass of the same steps with CUDA events around every "
                                  "layer-kernel launch on the launching stream",
                     "peak_kind": "bf16_tflops_sustained (%s)" % pk_kind,
                     "hw_tensor_tflops": hw_achieved, "hw_frac": (hw_achieved / hw_peak) if hw_achieved else None,
                     "hw_peak": hw_peak, "hw_peak_dtype": dt_of_mode, "hw_peak_ratio_to_bf16": ratio,
                     "hw_peak_ratio_kind": ratio_kind, "dtype_probe_tflops": dtype_rates},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_baselines and not secondary and Dref is not None:
        # baseline (i): plain FP32 recursion with torch.matmul, TF32 off, the
        # same table; baseline (ii): FP64 eigendecomposition on the GPU
        th_tab, b0_tab, m0_tab, al_tab = ms.table(int(rec["model"]))
        tab = ms.tables[int(rec["model"])]
        th_ent = tab.get("theta_entropy")
        emin, emax = float(rec["e_min"]), float(rec["e_max"])
        out = {}

        def fp32_step():
            out["r"] = plain_fp32_recursion(Hm, mu, kT, [tuple(r) for r in th_tab], b0_tab, m0_tab, al_tab,
                                            emin, emax, th_ent)

        fp32_step()
        t32 = cuda_time(fp32_step, 2)
        D32, S32 = out["r"]
        err32 = float((D32.double() - Dref).abs().max())
        del D32, out
        torch.cuda.empty_cache()
        t64 = cuda_time(lambda: eig_reference_gpu(Hm, kT, n, mu), 1)
        result["baselines"] = {
            "plain_fp32_recursion": {"solves_per_s": 1 / t32, "max_abs_D_minus_Dref": err32,
                                     "abs_S_minus_Sref_per_n": abs(S32 - Sref) / n,
                                     "math": "torch.matmul fp32, allow_tf32=False, same tables"},
            "fp64_eigh_gpu": {"solves_per_s": 1 / t64, "how": "torch.linalg.eigh float64 + V f V^T + S"},
            "speedup_vs_fp32_recursion": value / world * t32,
            "speedup_vs_fp64_eigh": value / world * t64,
        }
    del Dref
    torch.cuda.empty_cache()
    return result


# ---------------------------------------------------------------------------
# our arm: the ragged batch
# ---------------------------------------------------------------------------
def run_ragged(args, ft, world, rank, local, secondary=False):
    """The ragged batch (this rank's share of it, split by sum n^3): one
    grouped launch per layer for all instances and both chains, recorded into
    a CUDA graph and timed as graph replays."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import workloads as wl
    batch = wl.ragged_batch(args.batch, args.seed)
    mine = partition_by_work([b["n"] for b in batch], world)[rank]
    sub = [batch[b] for b in mine]
    Hs = [b["H"] for b in sub]
    ns = [b["n"] for b in sub]
    flat, _ = wl.pack_batch(Hs)
    Hd = torch.from_numpy(flat).cuda()
    ms = ft.ModelSet.from_json(table_paths(args))
    flags = flags_of(args, ft)
    mus, kTs = [b["mu"] for b in sub], [b["kT"] for b in sub]
    solver = ft.Solver(ns, mus, kTs, ms, mode=args.mode, want=3, flags=flags)
    if args.shape == "auto":
        shape, ms_single, ms_pair = solver.autotune(Hd, reps=1)
    else:
        shape, ms_single, ms_pair = solver.tile_shape()[0], None, None
    for _ in range(max(3, args.warmup)):
        solver.run(Hd)
    torch.cuda.synchronize()
    rec = solver.records()
    valid = rec["status"] == 0
    c0 = ft.kernel_launch_count()
    solver.run(Hd)
    per_run = ft.kernel_launch_count() - c0
    t_eager = cuda_time(lambda: solver.run(Hd), 3)
    graph = solver.graph(Hd)
    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: graph replays of the whole hot path ----
    steps = args.steps
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(steps):
            graph.replay()
        ev1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    value, t_step = aggregate(ev0.elapsed_time(ev1) / 1000.0 / steps, world, float(valid.sum()), device="cuda")

    # ---- layer times (second pass, eager, CUDA events around each layer launch) ----
    ft.profile_layers(True)
    ft.profile_read()
    for _ in range(3):
        solver.run(Hd)
    torch.cuda.synchronize()
    layer_ms, layer_n = ft.profile_read()
    ft.profile_layers(False)
    layers = rec["layers"]
    n3 = np.array(ns, dtype=np.float64) ** 3
    alg = float(np.sum((2.0 * n3 * layers)[valid]))            # both chains, L_b layers each
    lmax = int(layers.max())
    # per global layer in which instances are active (launches of layers before
    # the first active one leave at once)
    layer_avg = layer_ms / (3 * lmax) / 1000.0
    achieved = alg / lmax / layer_avg / 1e12 if layer_avg > 0 else None
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    # algorithmic bytes of one chain-layer of instance b: the state Z and A on
    # the upper triangle read and written (8 n^2 B), the next operands written
    # on the upper triangle (2 n^2 B) and this layer's read as full panels
    # (4 n^2 B); the layer moves them at a fraction of the HBM roof, well above
    # its fraction of the tensor roof
    n2 = np.array(ns, dtype=np.float64) ** 2
    alg_bytes = float(np.sum((2.0 * 14.0 * n2 * layers)[valid]))
    achieved_gbs = alg_bytes / lmax / layer_avg / 1e9 if layer_avg > 0 else None
    hbm_peak = pk.get("hbm_gbs")
    full_layer_bytes = float(np.sum((2.0 * 14.0 * n2)[valid]))
    cap = MEASURED_RAGGED_TRAFFIC.get((args.mode, args.batch, kernel_sha()))
    traffic = cap[0] / cap[1] * alg_bytes / lmax if cap else None

    # ---- accuracy on 32 instances spread over the sizes (the tests check all) ----
    errD, errS = 0.0, 0.0
    order = np.argsort(ns)
    picks = [int(order[i]) for i in np.linspace(0, len(ns) - 1, min(32, len(ns))).astype(int)]
    for b in picks:
        if not valid[b]:
            continue
        _, Dref, Sref, _, _ = eig_reference_gpu(torch.from_numpy(Hs[b]).cuda(), kTs[b], ns[b], mus[b])
        errD = max(errD, float((solver.matrix(b).double() - Dref).abs().max()))
        errS = max(errS, abs(float(solver.S[b]) - Sref) / ns[b])

    # ---- end to end through the API: H from pinned host memory, D, S and the
    # traces back to pinned host memory; two solvers alternate so that the
    # copies of one step overlap the other step's solve ----
    Hh = torch.from_numpy(flat).pin_memory()
    Dh = [torch.empty(solver.D.numel(), dtype=torch.float32).pin_memory() for _ in range(2)]
    Sh = [torch.empty(solver.S.numel(), dtype=torch.float64).pin_memory() for _ in range(2)]
    Th = [torch.empty(solver.trace.numel(), dtype=torch.float64).pin_memory() for _ in range(2)]
    Hdev = [torch.empty_like(Hd) for _ in range(2)]
    solvers = [solver, ft.Solver(ns, mus, kTs, ms, mode=args.mode, want=3, flags=flags)]
    solvers[1].run(Hd)                        # sets the second solver's kernel attributes
    torch.cuda.synchronize()
    comp = torch.cuda.current_stream()
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [[(Dh[k], solvers[k].D), (Sh[k], solvers[k].S), (Th[k], solvers[k].trace.view(-1))] for k in range(2)]
    overlapped_e2e(solvers, Hh, Hdev, outs, 2, comp, s_h2d, s_d2h)
    assert torch.equal(Dh[0], Dh[1]) and torch.equal(Dh[0], solver.D.cpu()), "end-to-end outputs differ"
    t_e2e = overlapped_e2e(solvers, Hh, Hdev, outs, max(3, steps // 2), comp, s_h2d, s_d2h)
    e2e_value, _ = aggregate(t_e2e, world, float(valid.sum()), device="cuda")
    Dh, Sh, Th = Dh[0], Sh[0], Th[0]
    del solvers, Hdev
    torch.cuda.empty_cache()

    result = {
        "metric": "ragged-batch instances/s (density + entropy) at <=1e-6 error", "value": value,
        "unit": "instances/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "fp16x2-split/fp32-accum" if args.mode == "fp16x2" else args.mode,
        "data": "synthetic", "config": ragged_config(args),
        "details": {"instances_this_rank": len(ns), "valid_instances_this_rank": int(valid.sum()),
                    "sum_n3_this_rank": float(np.sum(n3)), "global_layers": lmax,
                    "models_used": {int(m): int(np.sum(rec["model"] == m)) for m in np.unique(rec["model"])},
                    "tile_shape": {1: "256x256 CTA pairs", 0: "128x128 single CTAs", -1: "none"}[shape],
                    "autotune_ms": {"single": ms_single, "pair": ms_pair},
                    "timing": "CUDA-graph replays of one whole solve of the batch",
                    "eager_ms_per_step": t_eager * 1e3},
        "tflops_alg": alg / t_step / 1e12,
        "accuracy_sampled": {"instances": len(picks), "max_abs_D_minus_Dref": errD,
                             "max_abs_S_minus_Sref_per_n": errS},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_gbs / hbm_peak if achieved_gbs and hbm_peak else None,
                     "traffic": traffic,
                     "traffic_how": ("ncu dram bytes of one launch with every instance active, %.3g B against its "
                                     "%.3g algorithmic B, scaled to the mean launch by algorithmic bytes"
                                     % cap if cap else None),
                     "kernel": "layer_tc_kernel<%s>" % args.mode.upper(), "avg_layer_ms": layer_avg * 1e3,
                     "per_launch_alg_bytes": alg_bytes / lmax, "full_layer_alg_bytes": full_layer_bytes,
                     "peak_kind": "hbm_gbs (%s)" % pk_kind,
                     "tensor_achieved_tflops": achieved, "tensor_peak": peak,
                     "tensor_frac": achieved / peak if achieved else None,
                     "per_launch_alg_flops": alg / lmax,
                     "work_unit": "one global layer of every active instance and both chains: 14 n_b^2 B and "
                                  "n_b^3 flops per chain"},
        "e2e": {"value": e2e_value, "unit": "instances/s", "h2d_bytes_per_step": int(flat.nbytes),
                "d2h_bytes_per_step": int(Dh.numel() * 4 + Sh.numel() * 8 + Th.numel() * 8)},
        "gpu_launches": per_run * steps,
        "clocks": clk.summary(),
    }
    if not args.no_baselines and not secondary:
        # baseline (i): the plain FP32 recursion, one instance after the other
        # (torch.matmul, TF32 off), with each instance's own table and bounds
        def fp32_all():
            for b in range(len(ns)):
                if not valid[b]:
                    continue
                tab = ms.tables[int(rec["model"][b])]
                plain_fp32_recursion(torch.from_numpy(Hs[b]).cuda(), mus[b], kTs[b], [tuple(r) for r in tab["theta"]],
                                     tab["beta0"], tab["mu0"], tab["alpha"], float(rec["e_min"][b]),
                                     float(rec["e_max"][b]), tab.get("theta_entropy"))
        torch.backends.cuda.matmul.allow_tf32 = False
        fp32_all()
        t32 = cuda_time(fp32_all, 1)
        base = float(valid.sum()) / t32
        result["baselines"] = {"plain_fp32_recursion": {"instances_per_s": base,
                                                        "how": "per-instance torch.matmul fp32 loop, TF32 off"},
                               "speedup_vs_fp32_recursion": value / world / base}
    del graph
    torch.cuda.empty_cache()
    return result


FAMILY_TABLES = ["b100_L10", "b100_L12", "b100_L14", "max_b100_L8", "max_b100_L10", "max_b100_L12",
                  "skip22_b100_L10", "skip22_b100_L12", "skip22_b100_L14"]


def run_families(args, ft):
    """Layers against memory: the trained beta0 = 100 tables of the three
    families (Eq. mlsp2; Max-SP2; Skip-SP2 with two stored layers and two
    accumulators, run as its Max-SP2 embedding) on one n = 4096 lattice
    Hamiltonian, FP32 mode (the mode Max-SP2 tables run in), density and
    entropy.  Per table: its fitted max error on [0, 1], the measured time of
    a solve, the state planes a chain keeps, the workspace, the algorithmic
    HBM bytes of the layer epilogues (state planes read and written, FP32
    operands written) and the density error against the exact Fermi operator
    and against the table's own exact result."""
    import torch
    import workloads as wl
    dims = tuple(int(x) for x in args.dims.split(","))
    n = dims[0] * dims[1] * dims[2]
    kT = args.kT
    H = wl.lattice_3d(dims, args.seed)
    Hd = torch.from_numpy(H.ravel().copy()).cuda()
    torch.backends.cuda.matmul.allow_tf32 = False
    mu, Dref, Sref, eps, V = eig_reference_gpu(Hd.view(n, n), kT, n)
    rows = []
    plane = 4.0 * n * n
    for name in FAMILY_TABLES:
        path = os.path.join(TABLE_DIR, name + ".json")
        with open(path) as f:
            d = json.load(f)
        ms = ft.ModelSet.from_json([path])
        is_max = d.get("max") is not None
        L = int(d["L"])
        modes = ["fp32"] + ([] if is_max or L != 14 else ["fp16x2"])
        for mode in modes:
            # Lanczos bounds: the Gershgorin width of the noisy lattice would
            # put beta' beyond the beta0 = 100 tables' region at kT = 0.3
            solver = ft.Solver([n], [mu], [kT], ms, mode=mode, want=3, flags=ft.LANCZOS)
            for _ in range(max(3, args.warmup)):
                solver.run(Hd)
            torch.cuda.synchronize()
            rec = solver.records()[0]
            if rec["status"] != 0:
                raise SystemExit("%s: status %d" % (name, rec["status"]))
            t = cuda_time(lambda: solver.run(Hd), args.steps)
            D = solver.matrix(0).double()
            Drec, Srec = method_exact_gpu(eps, V, rec, ms.tables[0], mu)
            planes = L + 1 if is_max else 2
            # epilogue bytes per chain: Eq. mlsp2 reads and writes Z, A and
            # writes the operands (5 planes a layer); Max-SP2 layer k reads
            # k + 1 stored layers, writes one and the operands (k + 3)
            epi = sum((k + 3) if is_max else 5 for k in range(L)) * plane
            rows.append({"table": name, "family": ("Max-SP2" if name.startswith("max") else
                                                   "Skip-SP2 k=2 K=2 (as Max-SP2)" if name.startswith("skip22")
                                                   else "MLSP2"),
                         "mode": mode, "L": L, "max_err_fermi_fit": d["fit"]["max_err_fermi"],
                         "ms_per_solve": t * 1e3, "ms_per_layer": t * 1e3 / L,
                         "state_planes_per_chain": planes, "state_bytes": 2 * planes * plane,
                         "workspace_bytes": solver.ws_bytes, "epilogue_hbm_bytes": 2 * epi,
                         "err_D_vs_exact": float((D - Dref).abs().max()),
                         "err_D_vs_method_exact": float((D - Drec).abs().max()),
                         "err_S_vs_method_exact_per_n": abs(float(solver.S[0]) - Srec) / n})
            del solver, D, Drec
            torch.cuda.empty_cache()
    return {"metric": "family_layers_vs_memory", "unit": "ms/solve", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": "lattice %dx%dx%d (n=%d), kT=%g, mu at half filling, density+entropy"
                                   % (dims + (n, kT)), "tables": "beta0=100 families (trained by the library)",
                       "bounds": "lanczos"},
            "rows": rows}


def compact(res):
    """The headline keys of a secondary result."""
    keep = ("metric", "value", "unit", "ms_per_step", "tflops_alg", "config", "accuracy", "accuracy_sampled",
            "density_only", "e2e", "details")
    out = {k: res[k] for k in keep if k in res}
    r = res.get("roofline", {})
    out["roofline"] = {k: r.get(k) for k in ("bound", "unit", "achieved", "peak", "frac", "avg_layer_ms", "traffic",
                                             "tensor_frac")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
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
    if args.workload == "families":
        if rank == 0:
            print(json.dumps(run_families(args, ft)), flush=True)
        return
    if args.workload == "ragged":
        res = run_ragged(args, ft, world, rank, local)
    else:
        res = run_single(args, ft, world, rank, local)
    if rank == 0 and world == 1 and not args.no_baselines:
        res["cpu_baseline"] = cpu_baseline(args)
    if args.workload == "longrange" and world == 1 and not args.no_secondary:
        import copy
        sec = {}
        a2 = copy.copy(args)
        a2.workload, a2.refine, a2.steps = "ragged", None, max(5, args.steps // 2)
        sec["ragged_batch"] = compact(run_ragged(a2, ft, world, rank, local, secondary=True))
        a3 = copy.copy(args)
        a3.workload, a3.dims, a3.refine, a3.steps = "lattice", "16,16,16", None, max(5, args.steps // 2)
        sec["lattice_n4096"] = compact(run_single(a3, ft, world, rank, local, secondary=True))
        res["secondary"] = sec
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
