// (a7) Training kernels (Sec. II C): per-sample forward and reverse sweep of the
// scalar recursion (Eq. mlsp2, Skip-SP2 with one stored layer and one
// accumulator, or Max-SP2; each also under the entropy expansion of Eqs.
// entropy expansion / entropy expansion-s), and the FP64 reductions of one
// Levenberg-Marquardt iteration.
//
// Layout: the augmented Jacobian M = [J | r] is stored parameter-major,
// M[j * ns + s] (column j of J contiguous over samples), j = 0..np-1 for
// the table entries (a_0, b_0, c_0, d_0, a_1, ...), j = np for the residual.
// The Gram matrix G = M^T M holds J^T J, J^T r and r^T r; it is reduced over
// fixed sample chunks and then over chunks in a fixed order (deterministic).
#include "ftsp2_internal.h"

namespace ftsp2 {

constexpr int kTrainMaxL = kMaxLayers;

__device__ __forceinline__ double target_value(int target, double x, double beta0, double mu0) {
    const double t = beta0 * (x - mu0);
    if (target == FTSP2_TARGET_ENTROPY) {
        const double at = fabs(t);
        const double e = exp(-at);
        return log1p(e) + at * e / (1.0 + e);
    }
    // increasing logistic 1/(1 + exp(-t)), evaluated without overflow
    if (t >= 0.0) return 1.0 / (1.0 + exp(-t));
    const double e = exp(t);
    return e / (1.0 + e);
}

template <bool WITH_J>
__global__ void __launch_bounds__(128) fwd_kernel(int target, double beta0, double mu0, int L, double alpha,
                                                  const __grid_constant__ ThetaParam thp,
                                                  const double* __restrict__ X, int ns,
                                                  double* __restrict__ R, double* __restrict__ M) {
    const double* th = thp.v;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double x = X[s];
    double xs[kTrainMaxL + 1];
    double xi = target == FTSP2_TARGET_ENTROPY ? alpha * (x - mu0) + mu0 : x;
    double A = 0.0;
    for (int i = 0; i < L; ++i) {
        xs[i] = xi;
        const double a = th[4 * i], b = th[4 * i + 1], c = th[4 * i + 2],
                     d = th[4 * i + 3];
        A = fma(d, xi, A);
        xi = fma(fma(a, xi, b), xi, c);
    }
    const double F = A + xi;
    double out = F, fac = 1.0;
    if (target == FTSP2_TARGET_ENTROPY) {
        const double k4 = 4.0 * 0.69314718055994530942;
        out = k4 * F * (1.0 - F);
        fac = k4 * (1.0 - 2.0 * F);
    }
    const double r = out - target_value(target, x, beta0, mu0);
    R[s] = r;
    if (!WITH_J) return;
    const int np = 4 * L;
    M[(size_t)np * ns + s] = r;
    double g = 1.0;
    for (int i = L - 1; i >= 0; --i) {
        const double a = th[4 * i], b = th[4 * i + 1], d = th[4 * i + 3];
        const double x_i = xs[i];
        M[(size_t)(4 * i + 0) * ns + s] = fac * g * x_i * x_i;
        M[(size_t)(4 * i + 1) * ns + s] = fac * g * x_i;
        M[(size_t)(4 * i + 2) * ns + s] = fac * g;
        M[(size_t)(4 * i + 3) * ns + s] = fac * x_i;
        g = fma(g, fma(2.0 * a, x_i, b), d);
    }
}

// Skip-SP2 with one stored layer and one accumulator (Sec. II A 3): th holds
// L rows (delta, alpha, beta, gamma) and the output row (A_0, gamma_L);
// u_i = delta_i + alpha_i x_i + beta_i A_i, A_{i+1} = A_i + gamma_i x_i,
// x_{i+1} = u_i^2, F = A_L + gamma_L x_L.  Reverse sweep with gx = dF/dx_i,
// gA = dF/dA_i: w = 2 u_i gx_{i+1} gives dF/d(delta, alpha, beta)_i =
// w (1, x_i, A_i), dF/dgamma_i = gA_{i+1} x_i, gx_i = w alpha_i + gA_{i+1}
// gamma_i, gA_i = w beta_i + gA_{i+1}; dF/dA_0 = gA_0, dF/dgamma_L = x_L.
// Columns j < 4L + 2 in that flattened order, the residual in column 4L + 2.
template <bool WITH_J>
__global__ void __launch_bounds__(128) fwd_skip_kernel(int target, double beta0, double mu0, int L, double alpha,
                                                       const __grid_constant__ ThetaParam thp,
                                                       const double* __restrict__ X, int ns,
                                                       double* __restrict__ R, double* __restrict__ M) {
    const double* th = thp.v;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double x = X[s];
    double xs[kTrainMaxL], As[kTrainMaxL], us[kTrainMaxL];
    double xi = target == FTSP2_TARGET_ENTROPY ? alpha * (x - mu0) + mu0 : x;
    double A = th[4 * L];
    for (int i = 0; i < L; ++i) {
        xs[i] = xi;
        As[i] = A;
        const double u = fma(th[4 * i + 2], A, fma(th[4 * i + 1], xi, th[4 * i]));
        us[i] = u;
        A = fma(th[4 * i + 3], xi, A);
        xi = u * u;
    }
    const double F = fma(th[4 * L + 1], xi, A);
    double out = F, fac = 1.0;
    if (target == FTSP2_TARGET_ENTROPY) {
        const double k4 = 4.0 * 0.69314718055994530942;
        out = k4 * F * (1.0 - F);
        fac = k4 * (1.0 - 2.0 * F);
    }
    const double r = out - target_value(target, x, beta0, mu0);
    R[s] = r;
    if (!WITH_J) return;
    const int np = 4 * L + 2;
    M[(size_t)np * ns + s] = r;
    M[(size_t)(4 * L + 1) * ns + s] = fac * xi;
    double gx = th[4 * L + 1], gA = 1.0;
    for (int i = L - 1; i >= 0; --i) {
        const double w = 2.0 * us[i] * gx;
        M[(size_t)(4 * i + 0) * ns + s] = fac * w;
        M[(size_t)(4 * i + 1) * ns + s] = fac * w * xs[i];
        M[(size_t)(4 * i + 2) * ns + s] = fac * w * As[i];
        M[(size_t)(4 * i + 3) * ns + s] = fac * gA * xs[i];
        const double gx_i = fma(w, th[4 * i + 1], gA * th[4 * i + 3]);
        gA = fma(w, th[4 * i + 2], gA);
        gx = gx_i;
    }
    M[(size_t)(4 * L) * ns + s] = fac * gA;
}

// Max-SP2 (Sec. II A 2, Eq. maxsp2) on the flat table th: for i < L the block
// (delta_i, gamma_i, theta_{i,0..i}) at off_i = i (i + 5) / 2, then (c, gamma_L);
// u_i = delta_i + sum_{j<=i} theta_{i,j} x_j, x_{i+1} = u_i^2,
// F = c + sum_{j<=L} gamma_j x_j.  Reverse sweep with g_j = dF/dx_j (from
// gamma_j; g_{i+1} is final once the layers after i are done):
// w = 2 u_i g_{i+1}, dF/d delta_i = w, dF/d theta_{i,j} = w x_j,
// g_j += w theta_{i,j}; dF/d gamma_j = x_j, dF/dc = 1.  Columns in the flat
// order, the residual after them.
constexpr int kTrainMaxMaxL = kMaxMaxLayers;

template <bool WITH_J>
__global__ void __launch_bounds__(128) fwd_max_kernel(int target, double beta0, double mu0, int L, double alpha,
                                                      const __grid_constant__ ThetaParam thp,
                                                      const double* __restrict__ X, int ns,
                                                      double* __restrict__ R, double* __restrict__ M) {
    const double* th = thp.v;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const double x = X[s];
    double xs[kTrainMaxMaxL + 1], us[kTrainMaxMaxL], g[kTrainMaxMaxL + 1];
    xs[0] = target == FTSP2_TARGET_ENTROPY ? alpha * (x - mu0) + mu0 : x;
    const int oc = L * (L + 5) / 2;            // offset of (c, gamma_L)
    double F = th[oc];
    for (int i = 0; i < L; ++i) {
        const int o = i * (i + 5) / 2;
        double u = th[o];
        for (int j = 0; j <= i; ++j) u = fma(th[o + 2 + j], xs[j], u);
        us[i] = u;
        xs[i + 1] = u * u;
        F = fma(th[o + 1], xs[i], F);
    }
    F = fma(th[oc + 1], xs[L], F);
    double out = F, fac = 1.0;
    if (target == FTSP2_TARGET_ENTROPY) {
        const double k4 = 4.0 * 0.69314718055994530942;
        out = k4 * F * (1.0 - F);
        fac = k4 * (1.0 - 2.0 * F);
    }
    const double r = out - target_value(target, x, beta0, mu0);
    R[s] = r;
    if (!WITH_J) return;
    const int np = oc + 2;
    M[(size_t)np * ns + s] = r;
    M[(size_t)oc * ns + s] = fac;
    M[(size_t)(oc + 1) * ns + s] = fac * xs[L];
    for (int j = 0; j < L; ++j) g[j] = th[j * (j + 5) / 2 + 1];
    g[L] = th[oc + 1];
    for (int i = L - 1; i >= 0; --i) {
        const int o = i * (i + 5) / 2;
        const double w = 2.0 * us[i] * g[i + 1];
        M[(size_t)o * ns + s] = fac * w;
        M[(size_t)(o + 1) * ns + s] = fac * xs[i];
        for (int j = 0; j <= i; ++j) {
            M[(size_t)(o + 2 + j) * ns + s] = fac * w * xs[j];
            g[j] = fma(w, th[o + 2 + j], g[j]);
        }
    }
}

cudaError_t launch_train_fwd_jac(int target, double beta0, double mu0, int L, double alpha, const ThetaParam& th,
                                 const double* dX, int ns, double* dR, double* dM, cudaStream_t s, int family) {
    if (family == FTSP2_FAMILY_MAX)
        fwd_max_kernel<true><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR, dM);
    else if (family == FTSP2_FAMILY_SKIP)
        fwd_skip_kernel<true><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR, dM);
    else fwd_kernel<true><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR, dM);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_train_residual(int target, double beta0, double mu0, int L, double alpha, const ThetaParam& th,
                                  const double* dX, int ns, double* dR, cudaStream_t s, int family) {
    if (family == FTSP2_FAMILY_MAX)
        fwd_max_kernel<false><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR,
                                                               nullptr);
    else if (family == FTSP2_FAMILY_SKIP)
        fwd_skip_kernel<false><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR,
                                                                nullptr);
    else fwd_kernel<false><<<(ns + 127) / 128, 128, 0, s>>>(target, beta0, mu0, L, alpha, th, dX, ns, dR, nullptr);
    count_launch();
    return cudaGetLastError();
}

// Gram matrix of the columns of M (m = np + 1 columns of ns samples):
// grid (tiles of 32 x 32 entries, sample chunks); each block writes a partial
// tile for its chunk; gram_reduce sums the chunks in order.
constexpr int GT = 32;
constexpr int GS = 32;

__global__ void __launch_bounds__(256) gram_partial_kernel(const double* __restrict__ M, int ns, int m, int chunk,
                                                           double* __restrict__ part) {
    const int nt = (m + GT - 1) / GT;
    const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
    if (tj < ti) return;                       // upper tiles only; mirrored in the reduction
    const int s0 = blockIdx.y * chunk, s1 = min(ns, s0 + chunk);
    __shared__ double Si[GS][GT + 1], Sj[GS][GT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of threads
    double acc[4] = {0, 0, 0, 0};
    for (int sb = s0; sb < s1; sb += GS) {
        for (int e = threadIdx.x; e < GS * GT; e += 256) {
            const int col = e / GS, smp = e % GS;
            const int s = sb + smp;
            const int ci = ti * GT + col, cj = tj * GT + col;
            Si[smp][col] = (s < s1 && ci < m) ? M[(size_t)ci * ns + s] : 0.0;
            Sj[smp][col] = (s < s1 && cj < m) ? M[(size_t)cj * ns + s] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < GS; ++k) {
            const double bj = Sj[k][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(Si[k][ty * 4 + u], bj, acc[u]);
        }
        __syncthreads();
    }
    const size_t mm = (size_t)m * m;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int gi = ti * GT + ty * 4 + u, gj = tj * GT + tx;
        if (gi < m && gj < m) part[blockIdx.y * mm + (size_t)gi * m + gj] = acc[u];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int m, int nchunks, double* __restrict__ G) {
    const size_t mm = (size_t)m * m;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        const int ii = min(i, j), jj = max(i, j);
        // only tiles with tile(ii) <= tile(jj) were written; (ii, jj) always is
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += part[c * mm + (size_t)ii * m + jj];
        G[e] = s;
    }
}

cudaError_t launch_train_gram(const double* dM, int ns, int np, double* dG, double* dScratch, int nchunks,
                              cudaStream_t s) {
    const int m = np + 1;
    const int nt = (m + GT - 1) / GT;
    const int chunk = (ns + nchunks - 1) / nchunks;
    dim3 grid(nt * nt, nchunks);
    gram_partial_kernel<<<grid, 256, 0, s>>>(dM, ns, m, chunk, dScratch);
    gram_reduce_kernel<<<64, 256, 0, s>>>(dScratch, m, nchunks, dG);
    count_launch(2);
    return cudaGetLastError();
}

// out[j] = sum_s M[j][s] * w_s with w_s = (2/h) ((rh_s - r_s)/h - sum_j' J[j'][s] v[j'])
// (geodesic-acceleration right-hand side J^T r_vv), or with plain w = v-sum
// when rh == nullptr (J v).  One block per 256-sample chunk, then an ordered
// reduction over chunks.
__global__ void __launch_bounds__(256) accel_partial_kernel(const double* __restrict__ M, int ns, int np,
                                                            const double* __restrict__ v, const double* __restrict__ rh,
                                                            double h, double* __restrict__ part) {
    __shared__ double w[256];
    const int s = blockIdx.x * 256 + threadIdx.x;
    double ws = 0.0;
    if (s < ns) {
        double jv = 0.0;
        for (int j = 0; j < np; ++j) jv = fma(M[(size_t)j * ns + s], v[j], jv);
        const double r = M[(size_t)np * ns + s];
        ws = (2.0 / h) * ((rh[s] - r) / h - jv);
    }
    w[threadIdx.x] = ws;
    __syncthreads();
    for (int j = threadIdx.x; j < np; j += 256) {
        double acc = 0.0;
        const int base = blockIdx.x * 256;
        for (int k = 0; k < 256 && base + k < ns; ++k) acc = fma(M[(size_t)j * ns + base + k], w[k], acc);
        part[(size_t)blockIdx.x * np + j] = acc;
    }
}

__global__ void accel_reduce_kernel(const double* __restrict__ part, int nblk, int np, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    double s = 0.0;
    for (int c = 0; c < nblk; ++c) s += part[(size_t)c * np + j];
    out[j] = s;
}

cudaError_t launch_train_accel(const double* dM, const double* dV, const double* dRh, double h, int ns, int np,
                               double* dPart, double* dOut, cudaStream_t s) {
    const int nblk = (ns + 255) / 256;
    accel_partial_kernel<<<nblk, 256, 0, s>>>(dM, ns, np, dV, dRh, h, dPart);
    accel_reduce_kernel<<<(np + 127) / 128, 128, 0, s>>>(dPart, nblk, np, dOut);
    count_launch(2);
    return cudaGetLastError();
}

// max |r_s| over samples: per-block maxima, then one block.
__global__ void absmax_kernel(const double* __restrict__ r, int ns, double* __restrict__ part) {
    __shared__ double sm[256];
    double m = 0.0;
    for (int s = blockIdx.x * 256 + threadIdx.x; s < ns; s += gridDim.x * 256) m = fmax(m, fabs(r[s]));
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

cudaError_t launch_train_absmax(const double* dR, int ns, double* dPart, double* dOut, cudaStream_t s) {
    absmax_kernel<<<64, 256, 0, s>>>(dR, ns, dPart);
    absmax_kernel<<<1, 256, 0, s>>>(dPart, 64, dOut);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace ftsp2
