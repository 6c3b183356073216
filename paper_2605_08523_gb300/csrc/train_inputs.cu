// Inputs of the coefficient training (a7) that the library builds itself
// (host code): the fixed sample set of Sec. II C 1 and the starting tables.
//
// Samples.  The fit runs on N scalar points of [0, 1] drawn once from a density
// that follows the derivative of the target (Sec. II C 1: sampling where the
// Fermi function is steep targets the maximum error), p(x) = 1 + |f'(x)| with
// f the increasing logistic 1/(1 + exp(-beta0 (x - mu0))) of the model frame.
// The CDF F of p is integrated by the trapezoid rule on 2,000,001 evenly
// spaced points and inverted by linear interpolation: x_s = F^-1(q_s), with
// q_s = (s + 1/2)/N (seed 0, deterministic) or q_s = (s + u_s)/N, u_s the top
// 53 bits of splitmix64(seed + s) scaled to [0, 1) (one point in each of the
// N equal-probability cells; splitmix64: Steele, Lea and Flood, OOPSLA 2014).
//
// Starting tables.  The paper starts from a "scaled and truncated SP2"
// sequence (Sec. II A 1).  Reading: the SP2 sequence for a known chemical
// potential (Eq. sp2-mu) at mu0, embedded as Eq. mlsp2 rows (Appendix C:
// X^2 -> (1, 0, 0, 0), 2X - X^2 -> (-1, 2, 0, 0)), with the affine
// contraction x -> mu0 + kappa (x - mu0) folded into layer 0 so that the slope
// at mu0 equals the target's beta0 / 4 (kappa = min(1, (beta0/4) / slope); the
// slope of the composition is the product of the layers' derivatives along
// the trajectory of mu0).  The one-term form (Eq. mlsp2_alt) starts from the
// same SP2 sequence written as squares, and Skip-SP2 from the Appendix
// embedding of the Eq. mlsp2 start.
#include <cmath>
#include <cstdint>
#include <vector>

#include "ftsp2_internal.h"

namespace ftsp2 {

static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void train_sample_grid(double beta0, double mu0, int N, uint64_t seed, double* x) {
    constexpr int kFine = 2000001;
    const double step = 1.0 / (double)(kFine - 1);
    const double kT = 1.0 / beta0;
    std::vector<double> g(kFine), p(kFine), cdf(kFine);
    for (int i = 0; i < kFine; ++i) g[i] = (double)i * step;
    g[kFine - 1] = 1.0;
    for (int i = 0; i < kFine; ++i) {
        // occupation of the level -x at chemical potential -mu0 (Eq. FD_Func),
        // i.e. the increasing logistic of x, evaluated without overflow
        const double t = (-g[i] - (-mu0)) / kT;
        double f;
        if (t > 0.0) {
            const double e = std::exp(-t);
            f = e / (1.0 + e);
        } else {
            f = 1.0 / (1.0 + std::exp(t));
        }
        const double fp = beta0 * f * (1.0 - f);
        p[i] = 1.0 + std::fabs(fp);
    }
    cdf[0] = 0.0;
    for (int i = 1; i < kFine; ++i) cdf[i] = cdf[i - 1] + 0.5 * (p[i] + p[i - 1]) * (g[i] - g[i - 1]);
    const double total = cdf[kFine - 1];
    for (int i = 0; i < kFine; ++i) cdf[i] /= total;
    for (int s = 0; s < N; ++s) {
        double u = 0.5;
        if (seed != 0) u = (double)(splitmix64(seed + (uint64_t)s) >> 11) * 0x1.0p-53;
        const double q = ((double)s + u) / (double)N;
        // largest j with cdf[j] <= q (cdf is strictly increasing from 0 to 1)
        int lo = 0, hi = kFine - 1;
        if (q >= cdf[kFine - 1]) {
            x[s] = g[kFine - 1];
            continue;
        }
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (cdf[mid] <= q) lo = mid;
            else hi = mid;
        }
        if (cdf[lo] == q) {
            x[s] = g[lo];
        } else {
            const double slope = (g[lo + 1] - g[lo]) / (cdf[lo + 1] - cdf[lo]);
            x[s] = slope * (q - cdf[lo]) + g[lo];
        }
    }
}

// Branch choices of Eq. sp2-mu from m = mu': +1 for X^2 when
// |m^2 - mu'| < |2m - m^2 - mu'|, else -1 for 2X - X^2.
static void sp2_branches(double mu_p, int L, std::vector<int>& sig) {
    sig.assign(L, 0);
    double m = mu_p;
    for (int i = 0; i < L; ++i) {
        const double sq = m * m, up = 2.0 * m - m * m;
        if (std::fabs(sq - mu_p) < std::fabs(up - mu_p)) {
            sig[i] = 1;
            m = sq;
        } else {
            sig[i] = -1;
            m = up;
        }
    }
}

void train_init_mlsp2(int L, double beta0, double mu0, double* th) {
    std::vector<int> sig;
    sp2_branches(mu0, L, sig);
    for (int i = 0; i < L; ++i) {
        th[4 * i + 0] = sig[i] > 0 ? 1.0 : -1.0;
        th[4 * i + 1] = sig[i] > 0 ? 0.0 : 2.0;
        th[4 * i + 2] = 0.0;
        th[4 * i + 3] = 0.0;
    }
    double m = mu0, slope = 1.0;
    for (int i = 0; i < L; ++i) {
        const double a = th[4 * i], b = th[4 * i + 1], c = th[4 * i + 2];
        slope *= 2.0 * a * m + b;
        m = a * m * m + b * m + c;
    }
    const double kappa = std::fmin(1.0, (beta0 / 4.0) / slope);
    const double sh = mu0 * (1.0 - kappa);
    const double a = th[0], b = th[1], c = th[2];
    th[0] = a * kappa * kappa;
    th[1] = 2.0 * a * kappa * sh + b * kappa;
    th[2] = a * sh * sh + b * sh + c;
}

void train_init_alt(int L, double mu0, double* alt) {
    // The state y is x or 1 - x; both SP2 branches are squares of y or y - 1:
    // x^2 = (0 + y)^2 (or (-1 + y)^2 when y = 1 - x), and
    // 1 - (2x - x^2) = (1 - x)^2 = (-1 + y)^2 (or y^2 when y = 1 - x); the
    // output row undoes a final y = 1 - x.
    std::vector<int> sig;
    sp2_branches(mu0, L, sig);
    bool flipped = false;
    for (int i = 0; i < L; ++i) {
        if (sig[i] > 0) {
            alt[2 * i] = flipped ? -1.0 : 0.0;
            flipped = false;
        } else {
            alt[2 * i] = flipped ? 0.0 : -1.0;
            flipped = true;
        }
        alt[2 * i + 1] = 0.0;
    }
    alt[2 * L] = flipped ? 1.0 : 0.0;
    alt[2 * L + 1] = flipped ? -1.0 : 1.0;
}

void mlsp2_to_skip(int L, const double* th, double* tab) {
    // Appendix (MLSP2 in Skip-SP2): a_i x^2 + b_i x + c_i = a_i (x + b_i/(2a_i))^2 + e_i,
    // e_i = c_i - b_i^2/(4 a_i); the square is the next layer's x~, whose
    // combination carries a_{i-1} and e_{i-1}, the accumulator weights
    // d_i a_{i-1}, and the constants collect in A_0.
    std::vector<double> e(L);
    for (int i = 0; i < L; ++i) e[i] = th[4 * i + 2] - th[4 * i + 1] * th[4 * i + 1] / (4.0 * th[4 * i]);
    for (int i = 0; i < L; ++i) {
        const double a = th[4 * i], b = th[4 * i + 1], d = th[4 * i + 3];
        if (i == 0) {
            tab[0] = b / (2.0 * a);
            tab[1] = 1.0;
            tab[2] = 0.0;
            tab[3] = d;
        } else {
            const double ap = th[4 * (i - 1)];
            tab[4 * i + 0] = e[i - 1] + b / (2.0 * a);
            tab[4 * i + 1] = ap;
            tab[4 * i + 2] = 0.0;
            tab[4 * i + 3] = d * ap;
        }
    }
    double s = 0.0;
    for (int i = 1; i < L; ++i) s += th[4 * i + 3] * e[i - 1];
    tab[4 * L + 0] = e[L - 1] + s;
    tab[4 * L + 1] = th[4 * (L - 1)];
    tab[4 * L + 2] = 0.0;
    tab[4 * L + 3] = 0.0;
}

}  // namespace ftsp2
