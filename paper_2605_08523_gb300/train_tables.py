"""Train coefficient tables on the GPU with the library's own trainer and write
them as JSON (usage: ``python -m paper_2605_08523_gb300.train_tables OUTDIR``).

Two groups of tables:

* ``entropy_b1500_L26``: an entropy table (theta_entropy, Sec. II B) for the
  26-layer Fermi table printed in the paper's Appendix A, started from those
  Fermi weights (the paper's own recipe for theta_entropy) with
  alpha = 0.842704;
* the training sweep of L in {16, 24, 32} layers at scaled temperatures
  kT0 in [0.005, 0.05] (beta0 in {20, 50, 100, 200}, mu0 = 1/3): a Fermi table
  from the SP2 initial guess, then an entropy table started from it;
* ``--alt``: tables of the one-term form (Eq. mlsp2_alt) at (beta0, L) =
  (1500, 26) and (100, 16), from the SP2 sequence in that form
  (ftsp2_train_coeffs_alt), with entropy tables started from them;
* ``--skip``: Skip-SP2 tables (one stored layer, one accumulator): (1500, 26)
  from the embedding of the printed table, (100, 16) from the embedding of
  the SP2 initial guess (ftsp2_train_coeffs_skip), with entropy tables;
* ``--families``: at beta0 = 100, tables of the three families at several
  depths for the layers-against-memory comparison: Eq. mlsp2 (L = 10, 12,
  14), Max-SP2 (L = 8, 10, 12; ftsp2_train_coeffs_max) and Skip-SP2 with two
  stored layers and two accumulators (L = 10, 12, 14;
  ftsp2_train_coeffs_skipk, stored with its Max-SP2 embedding, the form the
  layer kernels run), each with an entropy table started from it;
* ``--grid B:L,... [ITER] [--polish N]``: tables at the given (beta0, L)
  pairs, optionally with N further seeded LM passes per fit;
* ``--high``: tables at beta0 in {3000, 6000, 12000, 24000} with
  L = ceil(layer count (Eq. layer count)) + 2 layers, which ragged batches of
  rotated spectra need once the Gershgorin width inflates beta'.

Every fit uses the library's 1e5 fixed samples from p ~ 1 + |f'|
(ftsp2_train_samples, seed 0) and Levenberg-Marquardt with geodesic
acceleration (ftsp2_train_coeffs).  The max
error of each table is measured on a uniform grid of 2e6 points in [0, 1].
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

from . import training

ALPHA = 0.842704
MU0 = 1.0 / 3.0


def max_error(ft, target, beta0, mu0, theta, alpha, grid=2_000_001, family=0):
    """max |model - target| of a table on a uniform grid of [0, 1], evaluated
    by the library (ftsp2_train_residuals)."""
    import torch
    x = torch.linspace(0.0, 1.0, grid, dtype=torch.float64, device="cuda")
    r = ft.ftsp2_train_residuals(target, beta0, mu0, theta, x, alpha=alpha, family=family)
    return float(r.abs().max())


def fit(ft, target, beta0, L, init, iterations, alpha=1.0, nsamples=100_000):
    t0 = time.time()
    th, rep = training.train_table(ft, target, beta0, MU0, L, alpha=alpha, iterations=iterations,
                                   nsamples=nsamples, theta_init=init)
    rep["seconds"] = time.time() - t0
    rep["max_err_grid"] = max_error(ft, target, beta0, MU0, th, alpha)
    return th, rep


def main_high(outdir: str, iterations: int = 3000):
    import math
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    for beta0 in (3000.0, 6000.0, 12000.0, 24000.0):
        L = int(math.ceil(training.layer_count(beta0))) + 2
        th, rep = fit(ft, ft.TARGET_FERMI, beta0, L, None, iterations)
        ths, reps = fit(ft, ft.TARGET_ENTROPY, beta0, L, th, iterations, alpha=ALPHA)
        name = "b%d_L%d" % (int(beta0), L)
        out[name] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, theta=th.tolist(), theta_entropy=ths.tolist(),
                         fit=dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"],
                                  max_err_sp2_init=max_error(ft, ft.TARGET_FERMI, beta0, MU0,
                                                             training.sp2_init(L, beta0, MU0), 1.0),
                                  layer_count=training.layer_count(beta0)),
                         train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
        print(name, out[name]["fit"], flush=True)
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(out[name], f, indent=1)
    return out


def main_alt(outdir: str, iterations: int = 3000):
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    for beta0, L in ((1500.0, 26), (100.0, 16)):
        t0 = time.time()
        alt, rep = training.train_alt_table(ft, ft.TARGET_FERMI, beta0, MU0, L, iterations=iterations)
        rep["seconds"] = time.time() - t0
        th = ft.ftsp2_alt_to_mlsp2(alt)
        rep["max_err_grid"] = max_error(ft, ft.TARGET_FERMI, beta0, MU0, th, 1.0)
        t0 = time.time()
        alts, reps = training.train_alt_table(ft, ft.TARGET_ENTROPY, beta0, MU0, L, alpha=ALPHA,
                                              iterations=iterations, alt_init=alt)
        reps["seconds"] = time.time() - t0
        reps["max_err_grid"] = max_error(ft, ft.TARGET_ENTROPY, beta0, MU0, ft.ftsp2_alt_to_mlsp2(alts), ALPHA)
        name = "alt_b%d_L%d" % (int(beta0), L)
        out[name] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, form="one-term (Eq. mlsp2_alt)",
                         alt=alt.tolist(), alt_entropy=alts.tolist(),
                         fit=dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"]),
                         train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
        print(name, out[name]["fit"], flush=True)
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(out[name], f, indent=1)
    return out


def skip_max_error(target, beta0, mu0, tab, alpha, grid=400_001):
    """max |model - target| of a Skip-SP2 table on a uniform grid."""
    import paper_2605_08523_gb300 as ft
    return max_error(ft, target, beta0, mu0, tab, alpha, grid=grid, family=1)


def main_skip(outdir: str, iterations: int = 3000):
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    printed = ft.ModelSet().table(0)[0]
    for beta0, L, init in ((1500.0, 26, training.skip_from_mlsp2(printed)), (100.0, 16, None)):
        t0 = time.time()
        tab, rep = training.train_skip_table(ft, ft.TARGET_FERMI, beta0, MU0, L, iterations=iterations,
                                             skip_init=init)
        rep["seconds"] = time.time() - t0
        rep["max_err_grid"] = skip_max_error(ft.TARGET_FERMI, beta0, MU0, tab, 1.0)
        t0 = time.time()
        tabs, reps = training.train_skip_table(ft, ft.TARGET_ENTROPY, beta0, MU0, L, alpha=ALPHA,
                                               iterations=iterations, skip_init=tab)
        reps["seconds"] = time.time() - t0
        reps["max_err_grid"] = skip_max_error(ft.TARGET_ENTROPY, beta0, MU0, tabs, ALPHA)
        name = "skip_b%d_L%d" % (int(beta0), L)
        fit = dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"])
        if init is not None:
            fit["max_err_fermi_start"] = skip_max_error(ft.TARGET_FERMI, beta0, MU0, init, 1.0)
        out[name] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, family="Skip-SP2, one stored layer, one accumulator",
                         skip=tab.tolist(), skip_entropy=tabs.tolist(), fit=fit,
                         train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
        print(name, out[name]["fit"], flush=True)
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(out[name], f, indent=1)
    return out


def fit_polished(ft, target, beta0, L, init, iterations, alpha=1.0, polish=0):
    """fit(), then `polish` further LM passes of `iterations` each, every pass
    started from the previous one's table on the sample set of seed 1, 2, ...
    (the fixed set of one pass is a different quantile draw of the same
    density); the table with the smallest max error on the grid is kept."""
    th, rep = fit(ft, target, beta0, L, init, iterations, alpha=alpha)
    best_th, best_rep, best_pass = th, rep, 0
    for sd in range(1, polish + 1):
        t0 = time.time()
        th, rep = training.train_table(ft, target, beta0, MU0, L, alpha=alpha, iterations=iterations,
                                       theta_init=th, seed=sd)
        rep["seconds"] = time.time() - t0
        rep["max_err_grid"] = max_error(ft, target, beta0, MU0, th, alpha)
        if rep["max_err_grid"] < best_rep["max_err_grid"]:
            best_th, best_rep, best_pass = th, rep, sd
    best_rep = dict(best_rep, polish_passes=polish, kept_pass=best_pass)
    return best_th, best_rep


def grid_args(argv):
    """(outdir, [(beta0, L), ...], iterations, polish passes) of a command
    line ``OUT --grid B:L,B:L [ITER] [--polish N]`` (any order)."""
    spec = argv[argv.index("--grid") + 1]
    pairs = [(float(b), int(l)) for b, l in (x.split(":") for x in spec.split(","))]
    skip = {argv.index("--grid") + 1}
    npol = 0
    if "--polish" in argv:
        npol = int(argv[argv.index("--polish") + 1])
        skip.add(argv.index("--polish") + 1)
    pos = [a for i, a in enumerate(argv) if i > 0 and i not in skip and not a.startswith("--")]
    return (pos[0] if pos else "tables_out"), pairs, (int(pos[1]) if len(pos) > 1 else 3000), npol


def main_grid(outdir: str, specs, iterations: int = 3000, polish: int = 0):
    """Tables at given (beta0, L) pairs (``--grid 2250:30,3000:32``), each a
    Fermi table from the SP2 initial guess and an entropy table started from
    it, written like the ``--high`` tables; ``--polish N`` adds N seeded LM
    passes to each fit (fit_polished)."""
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    for beta0, L in specs:
        th, rep = fit_polished(ft, ft.TARGET_FERMI, beta0, L, None, iterations, polish=polish)
        ths, reps = fit_polished(ft, ft.TARGET_ENTROPY, beta0, L, th, iterations, alpha=ALPHA, polish=polish)
        name = "b%d_L%d" % (int(beta0), L)
        out[name] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, theta=th.tolist(), theta_entropy=ths.tolist(),
                         fit=dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"],
                                  max_err_sp2_init=max_error(ft, ft.TARGET_FERMI, beta0, MU0,
                                                             training.sp2_init(L, beta0, MU0), 1.0),
                                  layer_count=training.layer_count(beta0)),
                         train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
        print(name, out[name]["fit"], flush=True)
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(out[name], f, indent=1)
    return out


def main_families(outdir: str, iterations: int = 1000):
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    beta0 = 100.0
    for L in (10, 12, 14):
        th, rep = fit(ft, ft.TARGET_FERMI, beta0, L, None, iterations)
        ths, reps = fit(ft, ft.TARGET_ENTROPY, beta0, L, th, iterations, alpha=ALPHA)
        out["b100_L%d" % L] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, theta=th.tolist(),
                                   theta_entropy=ths.tolist(),
                                   fit=dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"]),
                                   train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
    for L in (8, 10, 12):
        t0 = time.time()
        p, rep = ft.ftsp2_train_coeffs_max(ft.TARGET_FERMI, beta0, MU0, L=L, iterations=iterations)
        rep["seconds"] = time.time() - t0
        pe, reps = ft.ftsp2_train_coeffs_max(ft.TARGET_ENTROPY, beta0, MU0, max_init=p, iterations=iterations,
                                             alpha=ALPHA)
        fitd = dict(max_err_fermi=max_error(ft, ft.TARGET_FERMI, beta0, MU0, p, 1.0, family=2),
                    max_err_entropy=max_error(ft, ft.TARGET_ENTROPY, beta0, MU0, pe, ALPHA, family=2))
        out["max_b100_L%d" % L] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, family="Max-SP2", max=p.tolist(),
                                       max_entropy=pe.tolist(), fit=fitd,
                                       train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
    k, K = 2, 2
    for L in (10, 12, 14):
        t0 = time.time()
        v, rep = ft.ftsp2_train_coeffs_skipk(ft.TARGET_FERMI, beta0, MU0, L, k, K, iterations=iterations)
        rep["seconds"] = time.time() - t0
        ve, reps = ft.ftsp2_train_coeffs_skipk(ft.TARGET_ENTROPY, beta0, MU0, L, k, K, skip_init=v,
                                               iterations=iterations, alpha=ALPHA)
        p, pe = ft.ftsp2_skipk_to_max(v, L, k, K), ft.ftsp2_skipk_to_max(ve, L, k, K)
        fitd = dict(max_err_fermi=max_error(ft, ft.TARGET_FERMI, beta0, MU0, p, 1.0, family=2),
                    max_err_entropy=max_error(ft, ft.TARGET_ENTROPY, beta0, MU0, pe, ALPHA, family=2))
        out["skip22_b100_L%d" % L] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, k=k, K=K,
                                          family="Skip-SP2, two stored layers, two accumulators (as Max-SP2)",
                                          skipk=v.tolist(), skipk_entropy=ve.tolist(), max=p.tolist(),
                                          max_entropy=pe.tolist(), fit=fitd,
                                          train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
    for name, d in out.items():
        print(name, d["fit"], flush=True)
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(d, f, indent=1)
    return out


def main(outdir: str, iterations: int = 800, quick: bool = False):
    import paper_2605_08523_gb300 as ft
    from .build import build
    build()
    os.makedirs(outdir, exist_ok=True)
    out = {}
    # entropy table for the printed Fermi table
    ms = ft.ModelSet()
    printed, b0, m0, _ = ms.table(0)
    th_s, rep_s = fit(ft, ft.TARGET_ENTROPY, b0, 26, printed, 4 * iterations, alpha=ALPHA)
    out["entropy_b1500_L26"] = dict(beta0=b0, mu0=m0, alpha=ALPHA, L=26, theta=printed.tolist(),
                                    theta_entropy=th_s.tolist(),
                                    fit=dict(max_err_fermi=max_error(ft, ft.TARGET_FERMI, b0, m0, printed, 1.0),
                                             max_err_entropy=rep_s["max_err_grid"],
                                             max_err_entropy_theta_fermi=max_error(ft, ft.TARGET_ENTROPY, b0, m0,
                                                                                   printed, ALPHA)),
                                    train=dict(entropy=rep_s, samples=100_000, density="1+|f'|"))
    print("entropy_b1500_L26", out["entropy_b1500_L26"]["fit"], flush=True)
    betas = [20.0, 200.0] if quick else [20.0, 50.0, 100.0, 200.0]
    for beta0 in betas:
        for L in (16, 24, 32):
            th, rep = fit(ft, ft.TARGET_FERMI, beta0, L, None, iterations)
            ths, reps = fit(ft, ft.TARGET_ENTROPY, beta0, L, th, iterations, alpha=ALPHA)
            name = "b%d_L%d" % (int(beta0), L)
            out[name] = dict(beta0=beta0, mu0=MU0, alpha=ALPHA, L=L, theta=th.tolist(), theta_entropy=ths.tolist(),
                             fit=dict(max_err_fermi=rep["max_err_grid"], max_err_entropy=reps["max_err_grid"],
                                      max_err_sp2_init=max_error(ft, ft.TARGET_FERMI, beta0, MU0,
                                                                 training.sp2_init(L, beta0, MU0), 1.0),
                                      layer_count=training.layer_count(beta0)),
                             train=dict(fermi=rep, entropy=reps, samples=100_000, density="1+|f'|"))
            print(name, out[name]["fit"], flush=True)
    for name, d in out.items():
        with open(os.path.join(outdir, name + ".json"), "w") as f:
            json.dump(d, f, indent=1)
    return out


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    outdir = args[0] if args else "tables_out"
    if "--skip" in sys.argv:
        main_skip(outdir, iterations=int(args[1]) if len(args) > 1 else 3000)
    elif "--alt" in sys.argv:
        main_alt(outdir, iterations=int(args[1]) if len(args) > 1 else 3000)
    elif "--grid" in sys.argv:
        out, pairs, iters, npol = grid_args(sys.argv)
        main_grid(out, pairs, iterations=iters, polish=npol)
    elif "--families" in sys.argv:
        main_families(outdir, iterations=int(args[1]) if len(args) > 1 else 1000)
    elif "--high" in sys.argv:
        main_high(outdir, iterations=int(args[1]) if len(args) > 1 else 3000)
    else:
        main(outdir, iterations=int(args[1]) if len(args) > 1 else 800, quick="--quick" in sys.argv)
