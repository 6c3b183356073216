"""Writes tests/golden/max_table.json: a Max-SP2 table (Sec. II A 2) and a
Skip-SP2 table with k = 2 stored layers and K = 2 accumulators (Sec. II A 3),
both for beta0 = 100, mu0 = 1/3 and L = 12 layers, trained with the oracle's
Levenberg-Marquardt with geodesic acceleration (oracle.maxsp2.lm_fit and
oracle.maxsp2.skip_lm_fit) from the Appendix embeddings of the oracle's SP2
initial guess (oracle.train.init_from_sp2), and the Max-SP2 entropy table
trained from the Fermi table on the entropy target with alpha = 0.842704.
Calls only oracle/.  Run from the repository root:

    python tests/golden/make_max_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import maxsp2, skipsp2, train  # noqa: E402

BETA0, MU0, L, ALPHA = 100.0, 1.0 / 3.0, 12, 0.842704
K_STORED, K_ACC = 2, 2
NSAMPLES, ITERS = 20000, 600


def main():
    x = train.sample_grid(NSAMPLES, BETA0, MU0)
    th0 = train.init_from_sp2(L, BETA0, MU0)
    p, _ = maxsp2.lm_fit(maxsp2.mlsp2_to_max(th0), L, x, "fermi", BETA0, MU0, iters=ITERS, accel=True)
    err = maxsp2.max_error(p, L, "fermi", BETA0, MU0, grid=200_001)
    pe, _ = maxsp2.lm_fit(p, L, x, "entropy", BETA0, MU0, alpha=ALPHA, iters=ITERS // 2, accel=True)
    e_err = maxsp2.max_error(pe, L, "entropy", BETA0, MU0, alpha=ALPHA, grid=200_001)
    t0 = maxsp2.skip_from_skip1(skipsp2.from_mlsp2(th0), K_STORED, K_ACC, beta_extra=0.01)
    t, _ = maxsp2.skip_lm_fit(t0, "fermi", x, BETA0, MU0, iters=ITERS, accel=True)
    s_err = maxsp2.max_error(maxsp2.skip_to_max(t), L, "fermi", BETA0, MU0, grid=200_001)
    out = dict(beta0=BETA0, mu0=MU0, L=L, alpha=ALPHA, nsamples=NSAMPLES, iterations=ITERS,
               max=p.tolist(), max_err=err, max_entropy=pe.tolist(), max_err_entropy=e_err,
               skip22={k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in t.items()},
               skip22_max_err=s_err,
               source="oracle.maxsp2.lm_fit / skip_lm_fit (geodesic acceleration) from the embeddings of "
                      "oracle.train.init_from_sp2(L, beta0, mu0)")
    with open(os.path.join(HERE, "max_table.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("max-sp2 fermi %.3e entropy %.3e; skip-sp2 (2, 2) fermi %.3e" % (err, e_err, s_err))


if __name__ == "__main__":
    main()
