"""Writes tests/golden/skip_table.json: a Skip-SP2 table (one stored layer, one
accumulator) for beta0 = 100, mu0 = 1/3, L = 16, trained with the oracle's
Levenberg-Marquardt (oracle.skipsp2.lm_fit) from the Appendix embedding of the
oracle's SP2 initial guess (oracle.train.init_from_sp2), and its entropy table
trained from the Fermi table on the entropy target with alpha = 0.842704.
Calls only oracle/.  Run from the repository root:

    python tests/golden/make_skip_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import skipsp2, train  # noqa: E402

BETA0, MU0, L, ALPHA = 100.0, 1.0 / 3.0, 16, 0.842704
NSAMPLES, ITERS = 20000, 1000


def main():
    x = train.sample_grid(NSAMPLES, BETA0, MU0)
    t0 = skipsp2.from_mlsp2(train.init_from_sp2(L, BETA0, MU0))
    tab, _ = skipsp2.lm_fit(t0, x, "fermi", BETA0, MU0, iters=ITERS, accel=True)
    err = skipsp2.max_error(tab, "fermi", BETA0, MU0, grid=200_001)
    ent, _ = skipsp2.lm_fit(tab, x, "entropy", BETA0, MU0, alpha=ALPHA, iters=ITERS // 2, accel=True)
    e_err = skipsp2.max_error(ent, "entropy", BETA0, MU0, alpha=ALPHA, grid=200_001)
    out = dict(beta0=BETA0, mu0=MU0, L=L, alpha=ALPHA, nsamples=NSAMPLES, iterations=ITERS,
               skip=tab.tolist(), max_err=err, bound=2.0 * err, skip_entropy=ent.tolist(), max_err_entropy=e_err,
               max_abs_beta=float(abs(tab[:-1, 2]).max()),
               source="oracle.skipsp2.lm_fit (geodesic acceleration) from the embedding of "
                      "oracle.train.init_from_sp2(L, beta0, mu0)")
    with open(os.path.join(HERE, "skip_table.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("fermi max err %.3e, entropy max err %.3e, max|beta| %.3e" % (err, e_err, out["max_abs_beta"]))


if __name__ == "__main__":
    main()
