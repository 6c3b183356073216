"""Writes tests/golden/alt_table.json: a table of the one-term form (Eq.
mlsp2_alt) for beta0 = 100, mu0 = 1/3, L = 16, trained with the oracle's
Levenberg-Marquardt (oracle.altform.lm_fit) from the SP2 sequence at mu0, and
its entropy table trained from the Fermi table on the entropy target with
alpha = 0.842704.  Calls only oracle/.  Run from the repository root:

    python tests/golden/make_alt_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import altform, train  # noqa: E402

BETA0, MU0, L, ALPHA = 100.0, 1.0 / 3.0, 16, 0.842704
NSAMPLES, ITERS = 20000, 1000


def main():
    x = train.sample_grid(NSAMPLES, BETA0, MU0)
    alt, _ = altform.lm_fit(altform.sp2_alt(MU0, L), x, "fermi", BETA0, MU0, iters=ITERS, accel=True)
    err = altform.max_error(alt, "fermi", BETA0, MU0, grid=200_001)
    ent, _ = altform.lm_fit(alt, x, "entropy", BETA0, MU0, alpha=ALPHA, iters=ITERS // 2, accel=True)
    e_err = altform.max_error(ent, "entropy", BETA0, MU0, alpha=ALPHA, grid=200_001)
    out = dict(beta0=BETA0, mu0=MU0, L=L, alpha=ALPHA, nsamples=NSAMPLES, iterations=ITERS,
               alt=alt.tolist(), max_err=err, bound=2.0 * err, alt_entropy=ent.tolist(), max_err_entropy=e_err,
               source="oracle.altform.lm_fit (geodesic acceleration) from oracle.altform.sp2_alt(mu0, L)")
    with open(os.path.join(HERE, "alt_table.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("fermi max err %.3e, entropy max err %.3e" % (err, e_err))


if __name__ == "__main__":
    main()
