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

// Exclusive scan of one value per thread over the block (blockDim.x a multiple
// of 32, at most 1024): warp scans by shuffles, then the warp totals.
__device__ int block_exclusive_scan(int v, int& total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;      // inclusive warp prefix
    }
    __syncthreads();
    total = wsum[nw - 1];
    const int r = (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    __syncthreads();
    return r;
}

// Batches up to this many instances get their tiles in decreasing order of
// n (O(nb^2 / 1024) comparisons per thread of the one-block prep kernel).
constexpr int kTileSortMax = 2048;

// Per-instance tile ranges, then the tiles themselves.  A chain's table holds
// the instances one after the other, by decreasing n (ties by index) up to
// kTileSortMax instances, else in index order (thread t owns a contiguous
// chunk of instances; the chunk totals are scanned).  Warp w writes the tiles
// of instances w, w + 32, ..., its lanes stepping through the instance's list
// and decoding (I, J) from the position in the column-major triangle.
__device__ void block_exclusive_scan_fill(const ftsp2_instance* inst, int nb, int BM, int BN, int nchains,
                                          InstWork* iw, Tile* tiles, int table) {
    const int T = blockDim.x;
    const int chunk = (nb + T - 1) / T;
    const int b0 = min(nb, threadIdx.x * chunk);
    const int b1 = min(nb, b0 + chunk);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += tiles_of(inst[b].n, BM, BN);
    int chain_total;
    const int first = block_exclusive_scan(s, chain_total);
    if (nb <= kTileSortMax) {
        // instances by decreasing order n (ties by index): the units of a
        // layer launch take the tiles round-robin, so the long-K tiles are
        // dealt first and every unit's last tiles are short ones
        for (int b = b0; b < b1; ++b) {
            const int nself = inst[b].n, cnt = tiles_of(nself, BM, BN);
            int before = 0;
            for (int q = 0; q < nb; ++q) {
                const int nq = inst[q].n;
                if (nq > nself || (nq == nself && q < b)) before += tiles_of(nq, BM, BN);
            }
            for (int c = 0; c < nchains; ++c) {
                iw[b].tile_start[table][c] = c * chain_total + before;
                iw[b].tile_count[table][c] = cnt;
            }
        }
    } else {
        for (int c = 0; c < nchains; ++c) {
            int pos = c * chain_total + first;
            for (int b = b0; b < b1; ++b) {
                const int cnt = tiles_of(inst[b].n, BM, BN);
                iw[b].tile_start[table][c] = pos;
                iw[b].tile_count[table][c] = cnt;
                pos += cnt;
            }
        }
    }
    __syncthreads();
    const int q = BN / BM;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    for (int b = warp; b < nb; b += nw) {
        const int n = inst[b].n;
        const int nI = (n + BM - 1) / BM;
        const int cnt = iw[b].tile_count[table][0];
        for (int l = lane; l < cnt; l += 32) {
            int J = 0, rem = l;
            for (;;) {
                const int col = min(q * (J + 1), nI);
                if (rem < col) break;
                rem -= col;
                ++J;
            }
            for (int c = 0; c < nchains; ++c) tiles[iw[b].tile_start[table][c] + l] = Tile{b, rem, J, c};
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
    if (threadIdx.x == 0) {
        a.status[0] = 0;
        a.status[1] = 0x7fffffff;     // first global layer with an active instance (decide lowers it)
    }
    if (a.done) {
        const int cnt = a.done_layers * a.nb * kMaxChains;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) a.done[i] = 0;
    }
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
            // same pass, plus the FP32 copy the Lanczos matrix-vector products
            // read: instance b's slab of P x P floats, row pitch P (16-byte
            // aligned rows for vector loads).  Four loads are issued before
            // the four stores (a store may alias a later load as far as the
            // compiler knows), and the sums split as in the plain pass, so
            // both give the same bounds.
            float* hr = a.h32 + ((size_t)b * a.P + row) * a.P;
            for (; j + 96 < n; j += 128) {
                const double h0 = __ldg(Hr + j), h1 = __ldg(Hr + j + 32), h2 = __ldg(Hr + j + 64),
                             h3 = __ldg(Hr + j + 96);
                s0 += fabs(h0);
                s1 += fabs(h1);
                s2 += fabs(h2);
                s3 += fabs(h3);
                hr[j] = (float)h0;
                hr[j + 32] = (float)h1;
                hr[j + 64] = (float)h2;
                hr[j + 96] = (float)h3;
            }
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
    if (r.status == FTSP2_OK && r.model >= 0) {
        int first = sl[0];
        for (int c = 1; c < a.nchains; ++c) first = min(first, sl[c]);
        atomicMin(&a.status[1], first);
    }
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
// 32-byte store (sm_100+): dst 32-byte aligned.
__device__ __forceinline__ void st32(void* dst, const uint32_t* w) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// The operands of 16 consecutive elements of one row (idx0 % 16 == 0) in
// format FMT, as 32-byte vectors per plane; z == nullptr writes zeros.  One
// instantiation per format keeps only that format's planes in registers.
template <int FMT>
__device__ __forceinline__ void write_operand16_t(uint8_t* base, size_t plane_elems, size_t idx0, const float* z,
                                                  float scale) {
    constexpr int NPL = FMT == OP_F16X2 ? 2 : FMT == OP_BF16X3 ? 3 : FMT == OP_TF32X3 ? 2 : 1;
    constexpr int ESZ = (FMT == OP_F16X2 || FMT == OP_BF16X3) ? 2 : 4;
    constexpr int WORDS = 16 * ESZ / 4;
    uint32_t w[NPL][WORDS];
#pragma unroll
    for (int p = 0; p < NPL; ++p)
#pragma unroll
        for (int i = 0; i < WORDS; ++i) w[p][i] = 0u;
    if (z) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const float v = z[u];
            uint32_t o[NPL];
            if constexpr (FMT == OP_F16X2) {
                const float zs = v * scale;
                const __half h = __float2half_rn(zs);
                const __half l = __float2half_rn(zs - __half2float(h));
                o[0] = __half_as_ushort(h);
                o[1] = __half_as_ushort(l);
            } else if constexpr (FMT == OP_BF16X3) {
                const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
                const float r1 = v - __bfloat162float(b0);
                const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
                const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
                o[0] = __bfloat16_as_ushort(b0);
                o[1] = __bfloat16_as_ushort(b1);
                o[2] = __bfloat16_as_ushort(b2);
            } else if constexpr (FMT == OP_TF32X3) {
                uint32_t hb;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
                o[0] = hb;
                // the tensor core reads only the TF32 bits of the low part:
                // round it to TF32 here (unbiased) instead of letting them be cut
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(o[1]) : "f"(v - __uint_as_float(hb)));
            } else {
                o[0] = __float_as_uint(v);
            }
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
                if constexpr (ESZ == 2) w[p][u / 2] |= o[p] << (16 * (u & 1));
                else w[p][u] = o[p];
            }
        }
    }
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
        uint8_t* dst = base + ((size_t)p * plane_elems + idx0) * ESZ;
        st32(dst, w[p]);
        if constexpr (ESZ == 4) st32(dst + 32, w[p] + 8);
    }
}

__device__ __forceinline__ void write_operand16(int fmt, uint8_t* base, size_t plane_elems, size_t idx0,
                                                const float* z, float scale) {
    switch (fmt) {
        case OP_F16X2: write_operand16_t<OP_F16X2>(base, plane_elems, idx0, z, scale); break;
        case OP_BF16X3: write_operand16_t<OP_BF16X3>(base, plane_elems, idx0, z, scale); break;
        case OP_TF32X3: write_operand16_t<OP_TF32X3>(base, plane_elems, idx0, z, scale); break;
        default: write_operand16_t<OP_F32>(base, plane_elems, idx0, z, scale); break;
    }
}

// Layer-0 state and operands.  One CTA per (32-row band, instance, 512
// columns); lane = row of the band, each warp walks 16-column chunks of the
// band's columns in the instance's R x R square (R = n rounded up to the
// largest tile, 256, at most P):
// * Z_0 = z0 X, A = a0 X with X = H0 - mu0 I (times alpha for the entropy
//   chain; for Max-SP2 the stored layer x^_0 = X, z0 = 1, a0 = 0, and A is
//   the plane of x^_1, written by layer 0), in the blocked state layout, for
//   the rows below n and the chunks
//   that reach the upper triangle of the band's 32-row block (the only state
//   the layer epilogues read): four 512-byte runs per warp and chunk;
// * operands op0 Z_0 in the format of the instance's first layer (one parity),
//   zeros outside n x n in every format and parity a layer may read, as one
//   32-byte vector per lane and plane (row-major planes).  With `upper_only`
//   and a 16-bit first format (FP16X2, BF16X3) a real row r is written only
//   from the first column of its 256-row block on: the upper triangle plus the
//   diagonal blocks of either tile shape, the part a layer that loads the rest
//   as transposed panels reads.  Chunks left of that block are then skipped,
//   H included, when every chain of the instance takes this form.
// Z_0 is formed in FP64 and rounded once: scale * (mu - H_rr) on the diagonal,
// (-scale) * H_rc elsewhere (the same value as scale * (0 - H_rc)).
constexpr int kInitCols = 512;     // columns per init CTA

__global__ void __launch_bounds__(256) init_kernel(InitArgs a) {
    const int b = blockIdx.y;
    const ftsp2_instance in = a.inst[b];
    const int n = in.n, P = a.P;
    const int R = min(P, (n + 255) & ~255);
    const int band = blockIdx.x * 32;
    if (band >= R) return;
    const ftsp2_rescale_rec rec = a.rec[b];
    const bool ok = rec.status == FTSP2_OK && rec.model >= 0;
    const size_t base = (size_t)b * P * P;
    const int sl_packed = a.iw[b].start_layer;
    float alpha = 1.f, sc0 = 1.f, sc0S = 1.f, z0 = 1.f, a0 = 0.f, z0S = 1.f, a0S = 0.f, op0 = 1.f, op0S = 1.f;
    if (ok) {
        const DevModel& M = a.models[rec.model];
        alpha = (float)M.alpha;
        sc0 = M.scale0;
        sc0S = M.scale0S;
        z0 = M.z0;
        a0 = M.a0;
        z0S = M.z0S;
        a0S = M.a0S;
        op0 = M.op0;
        op0S = M.op0S;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cbeg = blockIdx.z * kInitCols, cend = min(R, cbeg + kInitCols);
    if (cbeg >= cend) return;
    const int r = band + lane;
    const bool row_in = r < n;
    const double* Hr = a.H + in.offset + (size_t)r * n;
    const double nscale = -rec.scale;
    // chains whose first layer reads the upper triangle plus diagonal blocks
    unsigned up_mask = 0u;
    for (int ch = 0; ch < a.nchains; ++ch) {
        const int start = (sl_packed >> (16 * ch)) & 0xffff;
        const bool ref = a.main_fmt != OP_F32 && start >= a.refine_from;
        const int f = ref ? a.refine_fmt : a.main_fmt;
        if (a.upper_only && (f == OP_F16X2 || f == OP_BF16X3)) up_mask |= 1u << ch;
    }
    const bool all_up = up_mask == (1u << a.nchains) - 1u;
    const int blk = band & ~255;               // first column of the band's 256-row block
    if (cend <= blk && all_up && band + 32 <= n) return;
    for (int cc = cbeg + warp * 16; cc < cend; cc += 8 * 16) {
        const bool low = cc + 16 <= blk;       // the chunk lies left of the diagonal block
        if (low && all_up && band + 32 <= n) continue;
        float z[16];
        if (ok && row_in && !(low && all_up)) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = cc + u;
                if (c < n) {
                    const double h = __ldg(Hr + c);
                    z[u] = (float)(r == c ? rec.scale * (in.mu - h) : nscale * h);
                } else {
                    z[u] = 0.f;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) z[u] = 0.f;
        }
        const bool inside = row_in && cc < n;        // the chunk holds elements of the n x n matrix
        const bool state = inside && cc + 15 >= band;
        for (int ch = 0; ch < a.nchains; ++ch) {
            const bool ent = a.chain_kind[ch] == CHAIN_ENTROPY;
            const float xs = ent ? alpha : 1.f;
            const float zf = (ent ? z0S : z0) * xs, af = (ent ? a0S : a0) * xs, of = ent ? op0S : op0;
            float zc[16], zo[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                zc[u] = zf * z[u];
                zo[u] = of * zc[u];      // the operands: zc itself unless op0 != 1 (Max-SP2)
            }
            if (state) {
#pragma unroll
                for (int blk = 0; blk < 2; ++blk) {
                    const size_t so = base + state_off(P, r, cc + 8 * blk);
                    float* Zs = a.Z[ch] + so;
                    float* As = a.A[ch] + so;
                    reinterpret_cast<float4*>(Zs)[0] = make_float4(zc[8 * blk], zc[8 * blk + 1], zc[8 * blk + 2], zc[8 * blk + 3]);
                    reinterpret_cast<float4*>(Zs + 128)[0] =
                        make_float4(zc[8 * blk + 4], zc[8 * blk + 5], zc[8 * blk + 6], zc[8 * blk + 7]);
                    reinterpret_cast<float4*>(As)[0] = make_float4(af * z[8 * blk], af * z[8 * blk + 1],
                                                                   af * z[8 * blk + 2], af * z[8 * blk + 3]);
                    reinterpret_cast<float4*>(As + 128)[0] = make_float4(af * z[8 * blk + 4], af * z[8 * blk + 5],
                                                                         af * z[8 * blk + 6], af * z[8 * blk + 7]);
                }
            }
            const size_t e0 = base + (size_t)r * P + cc;
            if (inside && low && ((up_mask >> ch) & 1u)) continue;
            if (inside) {
                // the values (zeros beyond n within the chunk) in the first layer's format
                const int start = (sl_packed >> (16 * ch)) & 0xffff;
                const bool ref = a.main_fmt != OP_F32 && start >= a.refine_from;
                if (ref) write_operand16(a.refine_fmt, a.OPR[ch][start & 1], a.plane_elems, e0, zo, 1.f);
                else write_operand16(a.main_fmt, a.OP[ch][start & 1], a.plane_elems, e0, zo, ent ? sc0S : sc0);
                if (cc + 15 >= n) {
                    // a chunk across the order: its padding columns must read as zero in
                    // every other format and parity too (its columns below n there are
                    // written by a layer before any layer reads them)
                    if (ref || (start & 1) != 0) write_operand16(a.main_fmt, a.OP[ch][0], a.plane_elems, e0, nullptr, 1.f);
                    if (ref || (start & 1) != 1) write_operand16(a.main_fmt, a.OP[ch][1], a.plane_elems, e0, nullptr, 1.f);
                    if (a.OPR[ch][0]) {
                        if (!ref || (start & 1) != 0)
                            write_operand16(a.refine_fmt, a.OPR[ch][0], a.plane_elems, e0, nullptr, 1.f);
                        if (!ref || (start & 1) != 1)
                            write_operand16(a.refine_fmt, a.OPR[ch][1], a.plane_elems, e0, nullptr, 1.f);
                    }
                }
            } else {
                // padding: zero in every format and parity a layer may read
                write_operand16(a.main_fmt, a.OP[ch][0], a.plane_elems, e0, nullptr, 1.f);
                write_operand16(a.main_fmt, a.OP[ch][1], a.plane_elems, e0, nullptr, 1.f);
                if (a.OPR[ch][0]) {
                    write_operand16(a.refine_fmt, a.OPR[ch][0], a.plane_elems, e0, nullptr, 1.f);
                    write_operand16(a.refine_fmt, a.OPR[ch][1], a.plane_elems, e0, nullptr, 1.f);
                }
            }
        }
    }
}

void launch_init(const InitArgs& a, int max_n, cudaStream_t s) {
    dim3 grid((a.P + 31) / 32, a.nb, (a.P + kInitCols - 1) / kInitCols);
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
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(FinalArgs a) {
    // one block per instance; each chain's partial sums are reduced by a
    // fixed assignment of slots to threads and a fixed tree, so the result
    // does not depend on scheduling
    const int b = blockIdx.x;
    if (b >= a.nb) return;
    __shared__ double s_tr[kFinThreads], s_sq[kFinThreads];
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
        for (int o = kFinThreads / 2; o > 0; o >>= 1) {
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
    finalize_kernel<<<a.nb, kFinThreads, 0, s>>>(a);
    count_launch();
}

}  // namespace ftsp2
