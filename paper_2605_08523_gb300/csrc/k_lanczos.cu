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
// Two launch shapes: batches whose instances all have n <= kLzSmallN run every
// step of an instance inside one CTA (vectors in shared memory, one CTA per
// SM so that the rows each CTA re-reads at every step can stay in L2); larger
// instances run each step as a multi-block matrix-vector launch plus an update
// launch.  The FP32 copy of H is stored per instance as a P x P slab with row
// pitch P, so every row starts 16-byte aligned.
// Reductions are in fixed order (deterministic).  The interval is not a
// rigorous enclosure; its safety terms (residual bound and the 1 % margin) are
// checked against the eigenvalues of the workload families in the tests.
#include <algorithm>

#include "ftsp2_internal.h"

namespace ftsp2 {

constexpr int kLzThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// fixed-order block sum of one double per thread (T threads)
template <int T = kLzThreads>
__device__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (t == 0) {
        for (int w = 0; w < T / 32; ++w) s += sh[w];
        sh[T / 32] = s;
    }
    __syncthreads();
    s = sh[T / 32];
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
        const float* Hr = a.H32 + ((size_t)b * a.P + row) * a.P;
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

// Small instances (every n <= kLzSmallN): one CTA runs all steps of one
// instance at a time, with the Lanczos vectors in shared memory and the first
// rows of H (as many as the dynamic shared memory holds) cached there too; the
// CTAs take the instances from a queue, largest order first (longest
// processing time first: a fixed round-robin split left the CTA with the most
// large instances running about twice the mean).  The launch asks for enough shared memory that
// one CTA runs per SM, so the rows of H that the resident CTAs re-read at every
// step (one instance each, at most kLzSmallN^2 floats) stay in L2 instead of
// streaming the whole batch from HBM 24 times.  Arithmetic as in the
// multi-block kernels: FP32 products and row sums, FP64 vectors, dot
// products and norms, reductions in a fixed order.
constexpr int kLzSmallN = 1024;
constexpr int kLzSmallThreads = 1024;
constexpr int kLzSmallCacheBytes = 160 * 1024;

// The queue of the small-instance kernel, in the partial-sum buffer (which
// only the multi-block path uses; nb RB doubles hold nb + 1 ints): queue[0]
// the next item (zeroed here), queue[1 + k] the instance of item k, by
// decreasing order n and then increasing index (the rank of b is the number
// of instances that come before it).  One thread per instance; O(nb^2)
// comparisons, a few microseconds up to kLzSortMax instances; larger batches
// keep their own order (the queue still balances the CTAs).
constexpr int kLzSortMax = 8192;
__device__ __forceinline__ int* lz_queue(const LanczosArgs& a) { return reinterpret_cast<int*>(a.part); }

__global__ void lanczos_queue_kernel(LanczosArgs a) {
    int* const queue = lz_queue(a);
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) queue[0] = 0;
    if (b >= a.nb) return;
    int rank = b;
    if (a.nb <= kLzSortMax) {
        const int nself = a.inst[b].n;
        rank = 0;
        for (int q = 0; q < a.nb; ++q) {
            const int nq = a.inst[q].n;
            rank += (nq > nself || (nq == nself && q < b)) ? 1 : 0;
        }
    }
    queue[1 + rank] = b;
}

__global__ void __launch_bounds__(kLzSmallThreads, 1) lanczos_small_kernel(LanczosArgs a) {
    __shared__ double vprev[kLzSmallN], vcur[kLzSmallN], w[kLzSmallN];
    __shared__ __align__(16) float v32[kLzSmallN];
    __shared__ double sh[kLzSmallThreads / 32 + 1];
    __shared__ int item;
    extern __shared__ float4 hcache4[];             // rows 0 .. rc - 1 of H (FP32), pitch pc
    float* const hcache = reinterpret_cast<float*>(hcache4);
    constexpr int NW = kLzSmallThreads / 32;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (;;) {
        // every thread has read `item` of the previous instance: the loop body
        // ends with a barrier
        if (t == 0) item = atomicAdd(lz_queue(a), 1);
        __syncthreads();
        const int k = item;
        if (k >= a.nb) break;
        const int b = lz_queue(a)[1 + k];
        const int n = a.inst[b].n;
        const float* Hb = a.H32 + (size_t)b * a.P * a.P;
        const int pc = (n + 3) & ~3;                 // cached row pitch (16-byte rows)
        const int rc = min(n, (int)(kLzSmallCacheBytes / (4 * pc)));
        for (int i = t; i < rc * pc; i += kLzSmallThreads) {
            const int r = i / pc, c = i - r * pc;
            hcache[i] = c < n ? Hb[(size_t)r * a.P + c] : 0.f;
        }
        // v_1 from the counter-based generator, v_0 = 0
        double s = 0.0;
        for (int i = t; i < n; i += kLzSmallThreads) {
            const double q = 2.0 * ((double)(splitmix64((unsigned long long)i) >> 11) * 0x1.0p-53) - 1.0;
            vcur[i] = q;
            vprev[i] = 0.0;
            s += q * q;
        }
        const double nrm = sqrt(block_sum<kLzSmallThreads>(s, sh));
        for (int i = t; i < n; i += kLzSmallThreads) {
            vcur[i] /= nrm;
            v32[i] = (float)vcur[i];
        }
        __syncthreads();
        double* ab = a.ab + (size_t)b * kLzSteps * 2;
        const int steps = min(n, kLzSteps);
        const int n4 = n >> 2;                       // whole float4 columns; the rest per lane
        double a1 = 0.0, b1 = 0.0, bprev = 0.0;
        int m = 0;
        bool stop = false;
        for (int j = 0; j < steps && !stop; ++j) {
            // w = H v_j - beta_{j-1} v_{j-1}: two rows per warp at a time,
            // 16-byte loads (rows of H are 16-byte aligned in both copies)
            const float4* v4 = reinterpret_cast<const float4*>(v32);
            for (int row = warp; row < n; row += 2 * NW) {
                const int row2 = row + NW;
                const bool two = row2 < n;
                const float* Ra = row < rc ? hcache + (size_t)row * pc : Hb + (size_t)row * a.P;
                const float* Rb = two ? (row2 < rc ? hcache + (size_t)row2 * pc : Hb + (size_t)row2 * a.P) : Ra;
                const float4* A4 = reinterpret_cast<const float4*>(Ra);
                const float4* B4 = reinterpret_cast<const float4*>(Rb);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll 4
                for (int q = lane; q < n4; q += 32) {
                    const float4 x = A4[q], y = B4[q], v = v4[q];
                    s0 = fmaf(x.x, v.x, s0);
                    s1 = fmaf(x.y, v.y, s1);
                    s2 = fmaf(x.z, v.z, s2);
                    s3 = fmaf(x.w, v.w, s3);
                    t0 = fmaf(y.x, v.x, t0);
                    t1 = fmaf(y.y, v.y, t1);
                    t2 = fmaf(y.z, v.z, t2);
                    t3 = fmaf(y.w, v.w, t3);
                }
                const int c = 4 * n4 + lane;
                if (c < n) {
                    s0 = fmaf(Ra[c], v32[c], s0);
                    t0 = fmaf(Rb[c], v32[c], t0);
                }
                float sa = (s0 + s1) + (s2 + s3), sb = (t0 + t1) + (t2 + t3);
                for (int o = 16; o > 0; o >>= 1) {
                    sa += __shfl_xor_sync(0xffffffffu, sa, o);
                    sb += __shfl_xor_sync(0xffffffffu, sb, o);
                }
                if (lane == 0) {
                    w[row] = (double)sa - bprev * vprev[row];
                    if (two) w[row2] = (double)sb - bprev * vprev[row2];
                }
            }
            __syncthreads();
            double p = 0.0;
            for (int i = t; i < n; i += kLzSmallThreads) p += w[i] * vcur[i];
            const double alpha = block_sum<kLzSmallThreads>(p, sh);
            p = 0.0;
            for (int i = t; i < n; i += kLzSmallThreads) {
                const double wi = w[i] - alpha * vcur[i];
                w[i] = wi;
                p += wi * wi;
            }
            const double beta = sqrt(block_sum<kLzSmallThreads>(p, sh));
            if (j == 0) {
                a1 = alpha;
                b1 = beta;
            }
            if (t == 0) {
                ab[2 * j] = alpha;
                ab[2 * j + 1] = beta;
            }
            m = j + 1;
            stop = beta <= 1e-12 * (fabs(a1) + b1 + 1.0);      // the same on every thread
            if (!stop) {
                for (int i = t; i < n; i += kLzSmallThreads) {
                    const double v = w[i] / beta;
                    vprev[i] = vcur[i];
                    vcur[i] = v;
                    v32[i] = (float)v;
                }
                bprev = beta;
            }
            __syncthreads();
        }
        if (t == 0) a.state[b] = m | (stop ? kLzStopped : 0);
        __syncthreads();
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
// per round; 8 rounds leave the edge within 33^-8 < 1e-12 of the bracket (the
// Gershgorin interval of T), far below the 1 % margin, and inside the 1e-10
// shift of the residual bound's inverse iteration
__device__ double edge_eigenvalue(const double* al, const double* be, int m, double lo, double hi, bool upper,
                                  int lane) {
    const int target = upper ? m : 1;
    double l = lo, h = hi;
    for (int it = 0; it < 8; ++it) {
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

void launch_lanczos(const LanczosArgs& a, int max_n, int sms, cudaStream_t s) {
    if (max_n <= kLzSmallN) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(lanczos_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kLzSmallCacheBytes);
            attr = true;
        }
        lanczos_queue_kernel<<<(a.nb + 255) / 256, 256, 0, s>>>(a);
        lanczos_small_kernel<<<std::min(a.nb, std::max(1, sms)), kLzSmallThreads, kLzSmallCacheBytes, s>>>(a);
        lanczos_bounds_kernel<<<(a.nb + 3) / 4, 128, 0, s>>>(a);
        count_launch(3);
        return;
    }
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
