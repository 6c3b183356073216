// Bandwidth-bound stages of the hot path:
//   prep       -- per-instance bookkeeping and the triangular tile tables
//   gershgorin -- (a1) spectral bounds, Appendix A: e_min = min_i(H_ii - R_i),
//                 e_max = max_i(H_ii + R_i), R_i = sum_{j != i} |H_ij|
//   decide     -- (a2) normalisation (Eqs. mu', beta'), flip (Eq. flip),
//                 validity (Eq. conditions), model choice (workflow step 4)
//   init       -- (a2) layer-0 state Z_0 = scale (mu I - H) (Eq. H0, centred),
//                 accumulators, first-layer tensor-core operands
//   finalize   -- (a4, a6) Tr D, ||D||_F^2 (Eq. tr(D^2)) and S (Eq. entropy
//                 expansion-s) from per-tile FP64 partial sums, in a fixed order
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ftsp2_internal.h"

namespace ftsp2 {

// ------------------------------------------------------------------------------
// prep: one block.  Initialises the bound keys and writes the tile tables.
// Tile (I, J) of an instance covers rows [128 I, 128 I + 128) and columns
// [BN J, BN J + BN); only tiles touching the upper triangle are listed
// (I < q (J + 1), q = BN / 128).  Chain-major order: all tiles of chain 0, then
// chain 1; inside a chain, instance by instance.
// ------------------------------------------------------------------------------
__device__ __forceinline__ int tiles_of(int n, int BM, int BN) {
    const int q = BN / BM;
    const int nI = (n + BM - 1) / BM;
    const int nJ = (n + BN - 1) / BN;
    int c = 0;
    for (int J = 0; J < nJ; ++J) c += min(q * (J + 1), nI);
    return c;
}

__device__ void block_exclusive_scan_fill(const ftsp2_instance* inst, int nb, int BM, int BN, int nchains,
                                          InstWork* iw, Tile* tiles, int table) {
    __shared__ int tot[1024];
    __shared__ int chain_total;
    const int T = blockDim.x;
    const int chunk = (nb + T - 1) / T;
    const int b0 = min(nb, threadIdx.x * chunk);
    const int b1 = min(nb, b0 + chunk);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += tiles_of(inst[b].n, BM, BN);
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < T; ++t) {
            const int v = tot[t];
            tot[t] = acc;
            acc += v;
        }
        chain_total = acc;
    }
    __syncthreads();
    const int q = BN / BM;
    for (int c = 0; c < nchains; ++c) {
        int pos = c * chain_total + tot[threadIdx.x];
        for (int b = b0; b < b1; ++b) {
            const int n = inst[b].n;
            const int nI = (n + BM - 1) / BM;
            const int nJ = (n + BN - 1) / BN;
            iw[b].tile_start[table][c] = pos;
            iw[b].tile_count[table][c] = tiles_of(n, BM, BN);
            for (int J = 0; J < nJ; ++J)
                for (int I = 0; I < min(q * (J + 1), nI); ++I) tiles[pos++] = Tile{b, I, J, c};
        }
    }
    __syncthreads();
}

__global__ void prep_kernel(SetupArgs a) {
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        a.iw[b].kmin = dkey(__longlong_as_double(0x7ff0000000000000ll));    // +inf
        a.iw[b].kmax = dkey(-__longlong_as_double(0x7ff0000000000000ll));   // -inf
        a.iw[b].nonfinite = 0;
        a.iw[b].start_layer = 0;
    }
    if (threadIdx.x == 0) *a.status = 0;
    if (a.tiles) block_exclusive_scan_fill(a.inst, a.nb, a.BM, a.BN, a.nchains, a.iw, a.tiles, 0);
    if (a.tiles_ref) block_exclusive_scan_fill(a.inst, a.nb, a.BM_ref, a.BN_ref, a.nchains, a.iw, a.tiles_ref, 1);
}

void launch_prep(const SetupArgs& a, cudaStream_t s) {
    prep_kernel<<<1, 1024, 0, s>>>(a);
    count_launch();
}

// ------------------------------------------------------------------------------
// gershgorin: one warp per row, coalesced FP64 loads, warp-shuffle sums, block
// min/max in shared memory, one atomic per block on order-preserving keys.
// ------------------------------------------------------------------------------
constexpr int kGWarps = 8;

__global__ void __launch_bounds__(kGWarps * 32) gershgorin_kernel(SetupArgs a) {
    const int b = blockIdx.y;
    const int n = a.inst[b].n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * kGWarps + warp;
    __shared__ double smin[kGWarps], smax[kGWarps];
    __shared__ int sbad[kGWarps];
    double lo = __longlong_as_double(0x7ff0000000000000ll), hi = -lo;
    int bad = 0;
    if (blockIdx.x * kGWarps >= n) return;     // whole block past the last row
    if (row < n) {
        const double* Hr = a.H + a.inst[b].offset + (size_t)row * n;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int j = lane;
        if (a.h32) {
            // same pass, plus the FP32 copy the Lanczos matrix-vector products read
            float* hr = a.h32 + a.inst[b].offset + (size_t)row * n;
            for (; j < n; j += 32) {
                const double h = __ldg(Hr + j);
                s0 += fabs(h);
                hr[j] = (float)h;
            }
        }
        for (; j + 96 < n; j += 128) {
            s0 += fabs(__ldg(Hr + j));
            s1 += fabs(__ldg(Hr + j + 32));
            s2 += fabs(__ldg(Hr + j + 64));
            s3 += fabs(__ldg(Hr + j + 96));
        }
        for (; j < n; j += 32) s0 += fabs(__ldg(Hr + j));
        double sum = (s0 + s1) + (s2 + s3);
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const double hii = __ldg(Hr + row);
        const double R = sum - fabs(hii);
        lo = hii - R;
        hi = hii + R;
        bad = !(isfinite(sum)) ? 1 : 0;
    }
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
        sbad[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = smin[0], h = smax[0];
        int bb = sbad[0];
        for (int w = 1; w < kGWarps; ++w) {
            l = fmin(l, smin[w]);
            h = fmax(h, smax[w]);
            bb |= sbad[w];
        }
        if (bb) atomicExch(&a.iw[b].nonfinite, 1);
        atomicMin(&a.iw[b].kmin, dkey(l));
        atomicMax(&a.iw[b].kmax, dkey(h));
    }
}

void launch_gershgorin(const SetupArgs& a, int max_n, cudaStream_t s) {
    dim3 grid((max_n + kGWarps - 1) / kGWarps, a.nb);
    gershgorin_kernel<<<grid, kGWarps * 32, 0, s>>>(a);
    count_launch();
}

// ------------------------------------------------------------------------------
// decide: one thread per instance (scalar decisions of Sec. III A).
// ------------------------------------------------------------------------------
__device__ __forceinline__ bool valid_region(double mup, double betap, double beta0, double mu0) {
    // spectrum of H0 inside [0, 1]: linear form of Eq. conditions
    const double s = betap / beta0;
    return (s * (0.0 - mup) + mu0 >= 0.0) && (s * (1.0 - mup) + mu0 <= 1.0);
}

// model preference (workflow step 4): smallest beta0 then fewest layers, or,
// with FTSP2_MIN_LAYERS, fewest (Fermi-chain) layers then smallest beta0
__device__ __forceinline__ bool better(const DevModel& m, const DevModel& cur, bool min_layers) {
    if (min_layers) return (m.L < cur.L) || (m.L == cur.L && m.beta0 < cur.beta0);
    return (m.beta0 < cur.beta0) || (m.beta0 == cur.beta0 && m.L < cur.L);
}

__global__ void decide_kernel(SetupArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nb) return;
    const ftsp2_instance in = a.inst[b];
    const bool min_layers = (a.flags & FTSP2_MIN_LAYERS) != 0;
    ftsp2_rescale_rec r;
    r.e_min = dunkey(a.iw[b].kmin);
    r.e_max = dunkey(a.iw[b].kmax);
    r.mu_p = 0.0;
    r.beta_p = 0.0;
    r.scale = 0.0;
    r.flip = 0;
    r.model = -1;
    r.status = FTSP2_OK;
    r.layers = 0;
    r.valid = 0;
    r.reserved = 0;
    int sl[kMaxChains] = {0, 0};
    if (a.iw[b].nonfinite || !isfinite(in.mu) || !isfinite(in.kT) || !(in.kT > 0.0) ||
        !isfinite(r.e_min) || !isfinite(r.e_max)) {
        r.status = FTSP2_E_NONFINITE;
    } else {
        const double beta = 1.0 / in.kT;
        int best = -1;
        if (r.e_max == r.e_min) {
            // H = cI: X0 = mu0 + (beta/beta0)(mu - c), no flip
            for (int m = 0; m < a.nmodels; ++m) {
                const double x = a.models[m].mu0 + (beta / a.models[m].beta0) * (in.mu - r.e_min);
                if (x >= 0.0 && x <= 1.0 && (best < 0 || better(a.models[m], a.models[best], min_layers))) best = m;
            }
            if (best >= 0) {
                r.model = best;
                r.valid = 1;
                r.scale = beta / a.models[best].beta0;
                r.mu_p = 0.0;
                r.beta_p = 0.0;
            } else {
                r.status = FTSP2_E_VALIDITY;
            }
        } else {
            const double W = r.e_max - r.e_min;
            double mup = (r.e_max - in.mu) / W;     // Eq. mu'
            double betap = W * beta;                 // Eq. beta'
            const int flip = mup > 0.5 ? 1 : 0;      // Eq. flip
            if (flip) mup = 1.0 - mup;
            for (int m = 0; m < a.nmodels; ++m)
                if (valid_region(mup, betap, a.models[m].beta0, a.models[m].mu0) &&
                    (best < 0 || better(a.models[m], a.models[best], min_layers)))
                    best = m;
            r.valid = best >= 0;
            if (best < 0 && (a.flags & FTSP2_CLAMP)) {
                best = 0;
                for (int m = 1; m < a.nmodels; ++m)
                    if (a.models[m].beta0 > a.models[best].beta0) best = m;
                const double b0 = a.models[best].beta0, m0 = a.models[best].mu0;
                double bmax = 1e300;
                if (mup > 0.0) bmax = fmin(bmax, m0 / mup * b0);
                if (mup < 1.0) bmax = fmin(bmax, (1.0 - m0) / (1.0 - mup) * b0);
                betap = fmin(betap, bmax);
            }
            r.mu_p = mup;
            r.beta_p = betap;
            r.flip = flip;
            if (best >= 0) {
                r.model = best;
                const double s = betap / (a.models[best].beta0 * W);
                r.scale = flip ? -s : s;
            } else {
                r.status = FTSP2_E_VALIDITY;
            }
        }
        if (r.model >= 0) {
            const DevModel& M = a.models[r.model];
            for (int c = 0; c < a.nchains; ++c) {
                const int Lc = a.chain_kind[c] == CHAIN_ENTROPY ? M.LS : M.L;
                sl[c] = a.Lmax - Lc;
            }
            r.layers = a.chain_kind[0] == CHAIN_ENTROPY ? M.LS : M.L;
        }
    }
    a.rec[b] = r;
    a.iw[b].start_layer = sl[0] | (sl[1] << 16);
}

void launch_decide(const SetupArgs& a, cudaStream_t s) {
    decide_kernel<<<(a.nb + 127) / 128, 128, 0, s>>>(a);
    count_launch();
}

// ------------------------------------------------------------------------------
// init: Z_0 = scale (mu I - H) on the padded P x P slab (zero outside n), the
// entropy chain's W_0 = alpha Z_0 (Eq. entropy expansion: y0 - mu0 =
// alpha (x0 - mu0)), A = 0, and the operands of each chain's first layer in the
// parity buffer of its start layer; the other parity buffer is zeroed so that
// padding rows and columns read as zeros in every layer.
// ------------------------------------------------------------------------------
__device__ __forceinline__ void write_operand(int fmt, uint8_t* base, size_t plane_elems, size_t idx,
                                              float z, float scale) {
    switch (fmt) {
        case OP_F32:
            reinterpret_cast<float*>(base)[idx] = z;
            break;
        case OP_TF32X3: {
            uint32_t hb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(z));
            const float h = __uint_as_float(hb);
            reinterpret_cast<float*>(base)[idx] = h;
            reinterpret_cast<float*>(base)[plane_elems + idx] = z - h;
            break;
        }
        case OP_BF16X3: {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(z);
            const float r1 = z - __bfloat162float(b0);
            const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(b1);
            const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
            __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base);
            p[idx] = b0;
            p[plane_elems + idx] = b1;
            p[2 * plane_elems + idx] = b2;
            break;
        }
        case OP_F16X2: {
            const float zs = z * scale;
            const __half h = __float2half_rn(zs);
            const __half l = __float2half_rn(zs - __half2float(h));
            __half* p = reinterpret_cast<__half*>(base);
            p[idx] = h;
            p[plane_elems + idx] = l;
            break;
        }
    }
}

__device__ __forceinline__ void zero_operand(int fmt, uint8_t* base, size_t plane_elems, size_t idx) {
    switch (fmt) {
        case OP_F32: reinterpret_cast<float*>(base)[idx] = 0.f; break;
        case OP_TF32X3:
            reinterpret_cast<float*>(base)[idx] = 0.f;
            reinterpret_cast<float*>(base)[plane_elems + idx] = 0.f;
            break;
        case OP_BF16X3: {
            uint16_t* p = reinterpret_cast<uint16_t*>(base);
            p[idx] = 0;
            p[plane_elems + idx] = 0;
            p[2 * plane_elems + idx] = 0;
            break;
        }
        case OP_F16X2: {
            uint16_t* p = reinterpret_cast<uint16_t*>(base);
            p[idx] = 0;
            p[plane_elems + idx] = 0;
            break;
        }
    }
}

__global__ void __launch_bounds__(256) init_kernel(InitArgs a) {
    const int b = blockIdx.y;
    const ftsp2_instance in = a.inst[b];
    const int n = in.n, P = a.P;
    const ftsp2_rescale_rec rec = a.rec[b];
    const bool ok = rec.status == FTSP2_OK && rec.model >= 0;
    const size_t base = (size_t)b * P * P;
    const int sl_packed = a.iw[b].start_layer;
    float alpha = 1.f, sc0 = 1.f, sc0S = 1.f, z0 = 1.f, a0 = 0.f, z0S = 1.f, a0S = 0.f;
    if (ok) {
        const DevModel& M = a.models[rec.model];
        alpha = (float)M.alpha;
        sc0 = M.scale0;
        sc0S = M.scale0S;
        z0 = M.z0;
        a0 = M.a0;
        z0S = M.z0S;
        a0S = M.a0S;
    }
    // The layers of this instance read rows and columns below n rounded up to
    // the largest tile (256), never the rest of the P x P slab: only that
    // square is initialised (padding zeroed).
    const int R = min(P, (n + 255) & ~255);
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const double* Hr = a.H + in.offset + (size_t)r * n;
        for (int c = threadIdx.x; c < R; c += blockDim.x) {
            const size_t e = base + (size_t)r * P + c;
            const size_t es = base + state_off(P, r, c);
            const bool inside = r < n && c < n;
            float z = 0.f;
            if (ok && inside) z = (float)(rec.scale * ((r == c ? in.mu : 0.0) - __ldg(Hr + c)));
            for (int ch = 0; ch < a.nchains; ++ch) {
                const bool ent = a.chain_kind[ch] == CHAIN_ENTROPY;
                // centred layer-0 input of the chain, then the family's layer-0 state
                const float xc = ent ? alpha * z : z;
                const float zc = (ent ? z0S : z0) * xc;
                a.Z[ch][es] = zc;
                a.A[ch][es] = (ent ? a0S : a0) * xc;
                if (inside) {
                    const int start = (sl_packed >> (16 * ch)) & 0xffff;
                    if (a.main_fmt != OP_F32 && start >= a.refine_from)
                        write_operand(a.refine_fmt, a.OPR[ch][start & 1], a.plane_elems, e, zc, 1.f);
                    else write_operand(a.main_fmt, a.OP[ch][start & 1], a.plane_elems, e, zc,
                                       ent ? sc0S : sc0);
                } else {
                    // padding: zero in every format and parity a layer may read
                    zero_operand(a.main_fmt, a.OP[ch][0], a.plane_elems, e);
                    zero_operand(a.main_fmt, a.OP[ch][1], a.plane_elems, e);
                    if (a.OPR[ch][0]) {
                        zero_operand(a.refine_fmt, a.OPR[ch][0], a.plane_elems, e);
                        zero_operand(a.refine_fmt, a.OPR[ch][1], a.plane_elems, e);
                    }
                }
            }
        }
    }
}

void launch_init(const InitArgs& a, int max_n, cudaStream_t s) {
    int gx = a.P < 2048 ? a.P : 2048;
    dim3 grid(gx, a.nb);
    init_kernel<<<grid, 256, 0, s>>>(a);
    count_launch();
}

// ------------------------------------------------------------------------------
// finalize: one block per instance.  Per chain the last layer left, per tile and
// per epilogue warp (kPartialSlots slots), two FP64 sums of the centred output G = A_L + Z_L:
// sum of the diagonal and sum of squares over the full matrix.  With
// D = G + f0 I (flipped: (1 - f0) I - G):
//   Tr D = n f0 + Tr G,  ||D||^2 = ||G||^2 + 2 f0 Tr G + n f0^2   (no flip)
//   Tr D = n (1 - f0) - Tr G, ||D||^2 = ||G||^2 - 2 (1 - f0) Tr G + n (1 - f0)^2
// and for the entropy chain F = G + g0 I:
//   S = 4 ln2 (Tr F - ||F||^2) = 4 ln2 (n g0 (1 - g0) + (1 - 2 g0) Tr G - ||G||^2).
// ------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) finalize_kernel(FinalArgs a) {
    // one block per instance; each chain's partial sums are reduced by a
    // fixed assignment of slots to threads and a fixed tree, so the result
    // does not depend on scheduling
    const int b = blockIdx.x;
    if (b >= a.nb) return;
    __shared__ double s_tr[256], s_sq[256];
    ftsp2_rescale_rec rec = a.rec[b];
    const int gstat = *a.status;
    const int n = a.inst[b].n;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int ch = 0; ch < a.nchains; ++ch) {
        double tr = 0.0, sq = 0.0;
        const int t0 = a.iw[b].tile_start[a.table][ch], tc = a.iw[b].tile_count[a.table][ch];
        for (int t = threadIdx.x; t < tc * kPartialSlots; t += blockDim.x) {
            tr += a.partials[(size_t)(t0 * kPartialSlots + t) * 2 + 0];
            sq += a.partials[(size_t)(t0 * kPartialSlots + t) * 2 + 1];
        }
        s_tr[threadIdx.x] = tr;
        s_sq[threadIdx.x] = sq;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                s_tr[threadIdx.x] += s_tr[threadIdx.x + o];
                s_sq[threadIdx.x] += s_sq[threadIdx.x + o];
            }
            __syncthreads();
        }
        tr = s_tr[0];
        sq = s_sq[0];
        __syncthreads();
        if (threadIdx.x != 0) continue;
        const bool ok = rec.status == FTSP2_OK && rec.model >= 0 && gstat == 0;
        if (a.chain_kind[ch] == CHAIN_FERMI) {
            double trD = qnan, frD = qnan;
            if (ok) {
                const double f0 = a.models[rec.model].f0;
                if (rec.flip) {
                    trD = n * (1.0 - f0) - tr;
                    frD = sq - 2.0 * (1.0 - f0) * tr + n * (1.0 - f0) * (1.0 - f0);
                } else {
                    trD = n * f0 + tr;
                    frD = sq + 2.0 * f0 * tr + n * f0 * f0;
                }
                if (!isfinite(trD) || !isfinite(frD)) rec.status = FTSP2_E_NONFINITE;
            }
            if (a.trace) {
                a.trace[2 * b + 0] = trD;
                a.trace[2 * b + 1] = frD;
            }
        } else {
            double S = qnan;
            if (ok) {
                const double g0 = a.models[rec.model].g0;
                S = 4.0 * 0.69314718055994530942 * (n * g0 * (1.0 - g0) + (1.0 - 2.0 * g0) * tr - sq);
                if (!isfinite(S)) rec.status = FTSP2_E_NONFINITE;
            }
            if (a.S) a.S[b] = S;
        }
    }
    if (threadIdx.x == 0) {
        if (gstat != 0 && rec.status == FTSP2_OK) rec.status = gstat;
        a.rec[b].status = rec.status;
    }
}

// ------------------------------------------------------------------------------
// One Newton-Raphson update of the chemical potential per instance (Sec. III A 4,
// Eqs. g, dg, delta_mu).  dD/dmu = +beta D (I - D) follows from the definition
// of D (the printed Eq. drho has the opposite sign), so
//   Delta mu = (N_occ - Tr D) / (beta (Tr D - ||D||_F^2)),
// limited to |Delta mu| <= W / 16 (W the Gershgorin width).  No step when
// |N_occ - Tr D| <= tol, when Tr D - ||D||_F^2 <= 0, or when the instance has no
// valid model.  One thread per instance.
// ------------------------------------------------------------------------------
__global__ void mu_update_kernel(MuArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nb) return;
    const ftsp2_rescale_rec rec = a.rec[b];
    if (rec.status != FTSP2_OK || rec.model < 0) return;
    const double trD = a.trace[2 * b], trD2 = a.trace[2 * b + 1];
    const double g = a.nocc[b] - trD;
    if (!(fabs(g) > a.tol)) return;
    const double kT = a.inst[b].kT;
    const double gp = (trD - trD2) / kT;
    if (!(gp > 0.0)) return;
    const double cap = (rec.e_max - rec.e_min) * (1.0 / 16.0);
    const double d = fmin(fmax(g / gp, -cap), cap);
    a.inst[b].mu += d;
    a.steps[b] += 1;
}

void launch_mu_update(const MuArgs& a, cudaStream_t s) {
    mu_update_kernel<<<(a.nb + 127) / 128, 128, 0, s>>>(a);
    count_launch();
}

void launch_finalize(const FinalArgs& a, cudaStream_t s) {
    finalize_kernel<<<a.nb, 256, 0, s>>>(a);
    count_launch();
}

}  // namespace ftsp2
