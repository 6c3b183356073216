// Spectral bounds tightened by a few Lanczos steps (FTSP2_LANCZOS).
//
// The Gershgorin interval of Appendix A over-estimates the spectrum of dense
// Hamiltonians by the row sums of |H_ij| (a dense 0.01 N(0,1) noise on an
// n = 4096 lattice, or a random rotation of a spectrum, widen it 5 to 12
// times).  W enters beta' = W beta (Eq. beta'), hence the beta0 a model needs,
// its layer count and the amplification of rounding.  Steps (per instance, all
// instances of a batch in the same launches):
//   start  v_1 = q / ||q||, q_i = 2 u_i - 1 with u_i the top 53 bits of
//          splitmix64(i) scaled to [0, 1) (Steele, Lea, Flood 2014);
//   k = min(n, kLzSteps) steps of the three-term recurrence, no
//          re-orthogonalisation:  w = H v_j - beta_{j-1} v_{j-1},
//          alpha_j = w . v_j,  w -= alpha_j v_j,  beta_j = ||w||,  v_{j+1} = w / beta_j,
//          stopping when beta_j <= 1e-12 (|alpha_1| + beta_1 + 1).  The products
//          H v_j read an FP32 copy of H and of v_j (written by the Gershgorin
//          pass and by the previous step) with FP32 row sums: this GPU's FP64
//          rate would bound an FP64 product, and the bounds need ~1e-6 relative
//          (they carry a 1 % margin); vectors, dot products and norms stay FP64;
//   bounds the extreme eigenvalues of the tridiagonal T_m (Sturm bisection) and
//          the residual bounds r = beta_m |s_m| of their Ritz vectors (inverse
//          iteration on T_m shifted just outside its spectrum):
//          lo = theta_min - r_min - delta, hi = theta_max + r_max + delta,
//          delta = 0.01 (theta_max - theta_min) + 1e-6 max(|theta_min|, |theta_max|),
//          intersected with Gershgorin (each end kept inside it).
// Reductions are in fixed order (deterministic).  The interval is not a
// rigorous enclosure; its safety terms (residual bound and the 1 % margin) are
// checked against the eigenvalues of the workload families in the tests.
#include "ftsp2_internal.h"

namespace ftsp2 {

constexpr int kLzThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// fixed-order block sum of one double per thread (kLzThreads threads)
__device__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (t == 0) {
        for (int w = 0; w < kLzThreads / 32; ++w) s += sh[w];
        sh[kLzThreads / 32] = s;
    }
    __syncthreads();
    s = sh[kLzThreads / 32];
    __syncthreads();
    return s;
}

__device__ __forceinline__ double* lz_vec(const LanczosArgs& a, int which, int b) {
    double* base = which == 0 ? a.V0 : (which == 1 ? a.V1 : a.W);
    return base + (size_t)b * a.P;
}

// v_1 from the counter-based generator; v_0 = 0; steps done = 0
__global__ void __launch_bounds__(kLzThreads) lanczos_start_kernel(LanczosArgs a) {
    __shared__ double sh[kLzThreads / 32 + 1];
    const int b = blockIdx.x;
    const int n = a.inst[b].n;
    double* v1 = lz_vec(a, 0, b);
    double* v0 = lz_vec(a, 1, b);
    float* v32 = a.V32 + (size_t)b * a.P;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kLzThreads) {
        const double u = (double)(splitmix64((unsigned long long)i) >> 11) * 0x1.0p-53;
        const double q = 2.0 * u - 1.0;
        v1[i] = q;
        v0[i] = 0.0;
        s += q * q;
    }
    const double nrm = sqrt(block_sum(s, sh));
    for (int i = threadIdx.x; i < n; i += kLzThreads) {
        v1[i] /= nrm;
        v32[i] = (float)v1[i];
    }
    if (threadIdx.x == 0) a.state[b] = 0;
}

__device__ __forceinline__ bool lz_active(const LanczosArgs& a, int b, int j, int n) {
    return j < n && !(a.state[b] & kLzStopped);
}

// w = H v_j - beta_{j-1} v_{j-1}; per block (kLzRows rows, one warp each) the
// partial sum of w . v_j
__global__ void __launch_bounds__(kLzRows * 32) lanczos_matvec_kernel(LanczosArgs a, int j) {
    const int b = blockIdx.y;
    const int n = a.inst[b].n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kLzRows + warp;
    __shared__ double sp[kLzRows];
    if (blockIdx.x * kLzRows >= n || !lz_active(a, b, j, n)) return;
    const double* vc = lz_vec(a, j & 1, b);
    const double* vp = lz_vec(a, (j + 1) & 1, b);
    const float* v32 = a.V32 + (size_t)b * a.P;
    double* w = lz_vec(a, 2, b);
    const double bprev = j > 0 ? a.ab[((size_t)b * kLzSteps + (j - 1)) * 2 + 1] : 0.0;
    double part = 0.0;
    if (row < n) {
        const float* Hr = a.H32 + a.inst[b].offset + (size_t)row * n;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int c = lane;
        for (; c + 96 < n; c += 128) {
            s0 = fmaf(__ldg(Hr + c), v32[c], s0);
            s1 = fmaf(__ldg(Hr + c + 32), v32[c + 32], s1);
            s2 = fmaf(__ldg(Hr + c + 64), v32[c + 64], s2);
            s3 = fmaf(__ldg(Hr + c + 96), v32[c + 96], s3);
        }
        for (; c < n; c += 32) s0 = fmaf(__ldg(Hr + c), v32[c], s0);
        float sf = (s0 + s1) + (s2 + s3);
        for (int o = 16; o > 0; o >>= 1) sf += __shfl_xor_sync(0xffffffffu, sf, o);
        const double wr = (double)sf - bprev * vp[row];
        if (lane == 0) w[row] = wr;
        part = wr * vc[row];
    }
    if (lane == 0) sp[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < kLzRows; ++r) t += sp[r];
        a.part[(size_t)b * a.RB + blockIdx.x] = t;
    }
}

// alpha_j, w -= alpha_j v_j, beta_j = ||w||, v_{j+1} = w / beta_j (into the
// buffer of v_{j-1}); one block per instance
__global__ void __launch_bounds__(kLzThreads) lanczos_update_kernel(LanczosArgs a, int j) {
    __shared__ double sh[kLzThreads / 32 + 1];
    const int b = blockIdx.x;
    const int n = a.inst[b].n;
    if (!lz_active(a, b, j, n)) return;
    const int nblk = (n + kLzRows - 1) / kLzRows;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kLzThreads) s += a.part[(size_t)b * a.RB + i];
    const double alpha = block_sum(s, sh);
    const double* vc = lz_vec(a, j & 1, b);
    double* vn = lz_vec(a, (j + 1) & 1, b);
    double* w = lz_vec(a, 2, b);
    s = 0.0;
    for (int i = threadIdx.x; i < n; i += kLzThreads) {
        const double wi = w[i] - alpha * vc[i];
        w[i] = wi;
        s += wi * wi;
    }
    const double beta = sqrt(block_sum(s, sh));
    double* ab = a.ab + (size_t)b * kLzSteps * 2;
    const double a1 = j == 0 ? alpha : ab[0];
    const double b1 = j == 0 ? beta : ab[1];
    const bool stop = beta <= 1e-12 * (fabs(a1) + b1 + 1.0);
    float* v32 = a.V32 + (size_t)b * a.P;
    if (!stop)
        for (int i = threadIdx.x; i < n; i += kLzThreads) {
            const double v = w[i] / beta;
            vn[i] = v;
            v32[i] = (float)v;
        }
    if (threadIdx.x == 0) {
        ab[2 * j] = alpha;
        ab[2 * j + 1] = beta;
        a.state[b] = (j + 1) | (stop ? kLzStopped : 0);
    }
}

// number of eigenvalues of the m x m tridiagonal (al, be) below x (Sturm)
__device__ int sturm_count(const double* al, const double* be, int m, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double off = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
        d = (al[i] - x) - (i > 0 ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// |last entry| of the unit eigenvector for the eigenvalue theta at the edge of
// the spectrum: inverse iteration with the shift just outside (sign = -1 below
// the smallest, +1 above the largest), where T - sigma I is definite and the
// tridiagonal elimination needs no pivoting
__device__ double edge_vector_last(const double* al, const double* be, int m, double theta, double sign,
                                   double scale) {
    double x[kLzSteps], c[kLzSteps], d[kLzSteps];
    const double sigma = theta + sign * 1e-10 * scale;
    for (int i = 0; i < m; ++i) x[i] = 1.0;
    for (int it = 0; it < 3; ++it) {
        // solve (T - sigma I) y = x (Thomas algorithm), y into x
        d[0] = al[0] - sigma;
        c[0] = x[0];
        for (int i = 1; i < m; ++i) {
            const double l = be[i - 1] / d[i - 1];
            d[i] = (al[i] - sigma) - l * be[i - 1];
            c[i] = x[i] - l * c[i - 1];
        }
        x[m - 1] = c[m - 1] / d[m - 1];
        for (int i = m - 2; i >= 0; --i) x[i] = (c[i] - be[i] * x[i + 1]) / d[i];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < m; ++i) x[i] /= nrm;
    }
    return fabs(x[m - 1]);
}

// eigenvalue of T_m at the lower (upper) edge by multisection: the 32 lanes
// count the eigenvalues below 32 points of the bracket, which shrinks 33-fold
// per round
__device__ double edge_eigenvalue(const double* al, const double* be, int m, double lo, double hi, bool upper,
                                  int lane) {
    const int target = upper ? m : 1;
    double l = lo, h = hi;
    for (int it = 0; it < 16; ++it) {
        const double x = l + (h - l) * (double)(lane + 1) / 33.0;
        const bool hit = sturm_count(al, be, m, x) >= target;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (mask == 0u) {
            l = __shfl_sync(0xffffffffu, x, 31);
        } else {
            const int k = __ffs(mask) - 1;
            const double xk = __shfl_sync(0xffffffffu, x, k);
            const double xk1 = __shfl_sync(0xffffffffu, x, k > 0 ? k - 1 : 0);
            if (k > 0) l = xk1;
            h = xk;
        }
    }
    return h;
}

// one warp per instance
__global__ void lanczos_bounds_kernel(LanczosArgs a) {
    __shared__ double sal[4][kLzSteps], sbe[4][kLzSteps];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int b = blockIdx.x * 4 + wi;
    if (b >= a.nb) return;
    const int m = a.state[b] & (kLzStopped - 1);
    if (m < 1) return;
    const double* ab = a.ab + (size_t)b * kLzSteps * 2;
    double* al = sal[wi];
    double* be = sbe[wi];
    for (int i = lane; i < m; i += 32) {
        al[i] = ab[2 * i];
        be[i] = ab[2 * i + 1];
    }
    __syncwarp();
    bool finite = true;
    double lo = 1e300, hi = -1e300;             // Gershgorin interval of T
    for (int i = 0; i < m; ++i) {
        finite = finite && isfinite(al[i]) && isfinite(be[i]);
        const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    if (!finite) return;                         // the Gershgorin bounds stay (and flag the input)
    const double tmin = edge_eigenvalue(al, be, m, lo, hi, false, lane);
    const double tmax = edge_eigenvalue(al, be, m, lo, hi, true, lane);
    if (lane != 0) return;
    const double scale = fmax(fabs(tmin), fabs(tmax)) + (tmax - tmin) + 1e-300;
    double rmin = 0.0, rmax = 0.0;
    const double blast = be[m - 1];
    if (m > 1 && blast > 0.0) {
        rmin = blast * edge_vector_last(al, be, m, tmin, -1.0, scale);
        rmax = blast * edge_vector_last(al, be, m, tmax, +1.0, scale);
    } else if (m == 1) {
        rmin = rmax = blast;
    }
    // 1 % of the Ritz spread, plus 1e-6 of the Ritz magnitude for the FP32 products
    const double delta = 0.01 * (tmax - tmin) + 1e-6 * fmax(fabs(tmin), fabs(tmax));
    const double elo = tmin - rmin - delta, ehi = tmax + rmax + delta;
    const double glo = dunkey(a.iw[b].kmin), ghi = dunkey(a.iw[b].kmax);
    if (!(isfinite(elo) && isfinite(ehi) && isfinite(glo) && isfinite(ghi))) return;
    // intersected with the Gershgorin interval, each end kept inside it
    a.iw[b].kmin = dkey(fmax(glo, fmin(elo, ghi)));
    a.iw[b].kmax = dkey(fmin(ghi, fmax(ehi, glo)));
}

static size_t lz_align(size_t x) { return (x + 1023) / 1024 * 1024; }

size_t lanczos_ws_bytes(int nb, int P) {
    const size_t vec = lz_align(sizeof(double) * (size_t)nb * P);
    const int RB = (P + kLzRows - 1) / kLzRows;
    return 3 * vec + lz_align(sizeof(float) * (size_t)nb * P) + lz_align(sizeof(double) * (size_t)nb * kLzSteps * 2) +
           lz_align(sizeof(double) * (size_t)nb * RB) + lz_align(sizeof(int) * (size_t)nb);
}

void lanczos_bind(LanczosArgs& a, uint8_t* ws, int nb, int P) {
    const size_t vec = lz_align(sizeof(double) * (size_t)nb * P);
    a.nb = nb;
    a.P = P;
    a.RB = (P + kLzRows - 1) / kLzRows;
    size_t off = 0;
    a.V0 = reinterpret_cast<double*>(ws + off);
    off += vec;
    a.V1 = reinterpret_cast<double*>(ws + off);
    off += vec;
    a.W = reinterpret_cast<double*>(ws + off);
    off += vec;
    a.V32 = reinterpret_cast<float*>(ws + off);
    off += lz_align(sizeof(float) * (size_t)nb * P);
    a.ab = reinterpret_cast<double*>(ws + off);
    off += lz_align(sizeof(double) * (size_t)nb * kLzSteps * 2);
    a.part = reinterpret_cast<double*>(ws + off);
    off += lz_align(sizeof(double) * (size_t)nb * a.RB);
    a.state = reinterpret_cast<int*>(ws + off);
}

void launch_lanczos(const LanczosArgs& a, int max_n, cudaStream_t s) {
    lanczos_start_kernel<<<a.nb, kLzThreads, 0, s>>>(a);
    count_launch();
    const int steps = max_n < kLzSteps ? max_n : kLzSteps;
    const dim3 mgrid((max_n + kLzRows - 1) / kLzRows, a.nb);
    for (int j = 0; j < steps; ++j) {
        lanczos_matvec_kernel<<<mgrid, kLzRows * 32, 0, s>>>(a, j);
        lanczos_update_kernel<<<a.nb, kLzThreads, 0, s>>>(a, j);
        count_launch(2);
    }
    lanczos_bounds_kernel<<<(a.nb + 3) / 4, 128, 0, s>>>(a);
    count_launch();
}

}  // namespace ftsp2
