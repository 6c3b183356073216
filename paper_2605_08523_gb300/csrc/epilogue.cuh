// Epilogue of one layer of the centred recursion, shared by the tensor-core
// and the CUDA-core layer kernels.  For an owned element (r, c), r <= c, with
// the constants of DevLayer:
//   xh = mul (Z_k^2)_{rc} + bp (Z_k)_{rc},   A' = A + d (Z_k)_{rc} + d2 xh,
//   Z_{k+1} = p xh + q A
// (centred Eq. mlsp2: Z_{k+1} = a_k Z_k^2 + (b_k + 2 a_k tau_k) Z_k,
// A' = A + d_k Z_k; centred Skip-SP2 with one stored layer and one
// accumulator: the square of the combination, then the next combination)
// then either the next layer's operands are written at (r, c) and (c, r), or,
// at the last layer, D = G + f0 I (Appendix A output, flipped as I - (A + X)
// when Eq. flip was used) is written and the FP64 partial sums of G are formed.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ftsp2_internal.h"

namespace ftsp2 {

// Is tile `t` active at global layer g?  Returns the instance's local layer k.
__device__ __forceinline__ bool tile_active_g(const LayerArgs& a, const Tile& t, int g, int& k) {
    const ftsp2_rescale_rec& rec = a.rec[t.inst];
    if (rec.status != FTSP2_OK || rec.model < 0) return false;
    const int start = (a.iw[t.inst].start_layer >> (16 * t.chain)) & 0xffff;
    k = g - start;
    return k >= 0;
}
// ... at this launch's (first) layer
__device__ __forceinline__ bool tile_active(const LayerArgs& a, const Tile& t, int& k) {
    return tile_active_g(a, t, a.gl, k);
}

// ----------------------------------------------------------------------------------
// Epilogue on one row segment of 16 columns (shared logic of the centred update).
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void store_operand(int fmt, uint8_t* base, size_t plane, size_t idx, float zs) {
    switch (fmt) {
        case OP_F32:
            reinterpret_cast<float*>(base)[idx] = zs;
            break;
        case OP_TF32X3: {
            uint32_t hb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(zs));
            const float h = __uint_as_float(hb);
            uint32_t lb;   // low part rounded to the TF32 bits the tensor core reads
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(zs - h));
            reinterpret_cast<float*>(base)[idx] = h;
            reinterpret_cast<float*>(base)[plane + idx] = __uint_as_float(lb);
            break;
        }
        case OP_BF16X3: {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(zs);
            const float r1 = zs - __bfloat162float(b0);
            const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
            const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
            __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base);
            p[idx] = b0;
            p[plane + idx] = b1;
            p[2 * plane + idx] = b2;
            break;
        }
        case OP_F16X2: {
            const __half h = __float2half_rn(zs);
            const __half l = __float2half_rn(zs - __half2float(h));
            __half* p = reinterpret_cast<__half*>(base);
            p[idx] = h;
            p[plane + idx] = l;
            break;
        }
    }
}

struct EpiCtx {
    int n, P, chain, kind, flip, last, next_fmt;
    float mul;            // multiplier of the product: a_k, times 2^(-2 e_k) for scaled FP16 operands
    size_t slab;          // b * P * P
    int64_t doff;         // D offset
    DevLayer L;
    double cdiag;         // f0 (or 1 - f0 when flipped) added on the diagonal of D
};

// Process row r, columns c0 .. c0 + W - 1 (c0 % 8 == 0, W % 4 == 0, c0 + W <= P) with
// accumulator values v[W].  Accumulates (diagonal sum, weighted square sum) of the
// centred output G into tr / sq at the last layer.
template <int W>
__device__ __forceinline__ void epi_segment(const LayerArgs& a, const EpiCtx& e, int r, int c0,
                                            const float* v, double& tr, double& sq) {
    if (r >= e.n) return;
    float* Zs = a.Z[e.chain] + e.slab;
    float* As = a.A[e.chain] + e.slab;
    float z[W], ac[W];
#pragma unroll
    for (int i = 0; i < W / 4; ++i) {
        const size_t o = state_off(e.P, r, c0 + 4 * i);
        const float4 zz = *reinterpret_cast<const float4*>(Zs + o);
        const float4 aa = *reinterpret_cast<const float4*>(As + o);
        z[4 * i + 0] = zz.x; z[4 * i + 1] = zz.y; z[4 * i + 2] = zz.z; z[4 * i + 3] = zz.w;
        ac[4 * i + 0] = aa.x; ac[4 * i + 1] = aa.y; ac[4 * i + 2] = aa.z; ac[4 * i + 3] = aa.w;
    }
    float zn[W], an[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const float xh = fmaf(e.mul, v[j], e.L.bp * z[j]);
        an[j] = fmaf(e.L.d2, xh, fmaf(e.L.d, z[j], ac[j]));
        zn[j] = e.last ? xh : fmaf(e.L.p, xh, e.L.q * ac[j]);
    }
    if (!e.last) {
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const size_t o = state_off(e.P, r, c0 + 4 * i);
            *reinterpret_cast<float4*>(Zs + o) = make_float4(zn[4 * i], zn[4 * i + 1], zn[4 * i + 2], zn[4 * i + 3]);
            *reinterpret_cast<float4*>(As + o) = make_float4(an[4 * i], an[4 * i + 1], an[4 * i + 2], an[4 * i + 3]);
        }
        uint8_t* ob = a.opw[e.chain];
        const float os = e.next_fmt == OP_F16X2 ? e.L.out_scale : 1.f;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int c = c0 + j;
            if (c < e.n && r <= c) {
                const float zs = zn[j] * os;
                store_operand(e.next_fmt, ob, a.plane_elems, e.slab + (size_t)r * e.P + c, zs);
                if (c != r) store_operand(e.next_fmt, ob, a.plane_elems, e.slab + (size_t)c * e.P + r, zs);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int c = c0 + j;
            if (c < e.n && r <= c) {
                const float g = fmaf(e.L.g, zn[j], an[j]);
                if (e.kind == CHAIN_FERMI && a.D) {
                    float dv;
                    if (e.flip) dv = (r == c ? (float)e.cdiag : 0.f) - g;
                    else dv = g + (r == c ? (float)e.cdiag : 0.f);
                    a.D[e.doff + (int64_t)r * e.n + c] = dv;
                    if (c != r) a.D[e.doff + (int64_t)c * e.n + r] = dv;
                }
                const double gd = (double)g;
                if (r == c) {
                    tr += gd;
                    sq += gd * gd;
                } else {
                    sq += 2.0 * gd * gd;
                }
            }
        }
    }
}

// Max-SP2 layer k (FP32 mode, CUDA-core layers only).  State plane j of the
// chain holds the centred stored layer x^_j = X_j - chi_j I (chi_j the layer
// values along the trajectory of mu0, sigma_k the combination's value there);
// the operands of layer k are the centred combination
// U^_k = sum_{j<=k} theta_{k,j} x^_j, and with v = (U^_k^2)_{rc}:
//   x^_{k+1} = v + 2 sigma_k U^_k          (bp = 2 sigma_k, mul = 1)
// is stored as plane k + 1 and the operands of layer k + 1,
// U^_{k+1} = sum_{j<=k+1} theta_{k+1,j} x^_j, are written at (r, c) and (c, r);
// the last layer forms G = sum_{j<=L} gamma_j x^_j instead (D = G + f0 I).
// U^_k is re-formed here from the planes in the order its operands were
// formed, so it equals the operand value the product used.
template <int W>
__device__ __forceinline__ void epi_segment_max(const LayerArgs& a, const EpiCtx& e, int r, int c0,
                                                const float* v, double& tr, double& sq) {
    if (r >= e.n) return;
    float* X = a.Z[e.chain] + e.slab;
    const int k1 = e.L.nplanes;                    // k + 1 stored layers are read
    const float* th = a.coef + e.L.coef;           // theta_{k,0..k}
    const float* tn = th + k1;                     // theta_{k+1,0..k+1}
    const float* gm = tn + k1 + 1;                 // gamma_{0..L} (last layer)
    float ui[W], un[W], g[W];
#pragma unroll
    for (int j = 0; j < W; ++j) ui[j] = un[j] = g[j] = 0.f;
    for (int p = 0; p < k1; ++p) {
        const float tk = th[p], tq = tn[p], gp = e.last ? gm[p] : 0.f;
        const float* Xp = X + (size_t)p * a.plane_elems;
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const float4 xx = *reinterpret_cast<const float4*>(Xp + state_off(e.P, r, c0 + 4 * i));
            const float xv[4] = {xx.x, xx.y, xx.z, xx.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ui[4 * i + q] = fmaf(tk, xv[q], ui[4 * i + q]);
                un[4 * i + q] = fmaf(tq, xv[q], un[4 * i + q]);
                g[4 * i + q] = fmaf(gp, xv[q], g[4 * i + q]);
            }
        }
    }
    float xn[W];
#pragma unroll
    for (int j = 0; j < W; ++j) xn[j] = fmaf(e.mul, v[j], e.L.bp * ui[j]);
    if (!e.last) {
        float* Xn = X + (size_t)k1 * a.plane_elems;
#pragma unroll
        for (int i = 0; i < W / 4; ++i)
            *reinterpret_cast<float4*>(Xn + state_off(e.P, r, c0 + 4 * i)) =
                make_float4(xn[4 * i], xn[4 * i + 1], xn[4 * i + 2], xn[4 * i + 3]);
        const float tl = tn[k1];
        uint8_t* ob = a.opw[e.chain];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int c = c0 + j;
            if (c < e.n && r <= c) {
                const float zs = fmaf(tl, xn[j], un[j]);
                store_operand(e.next_fmt, ob, a.plane_elems, e.slab + (size_t)r * e.P + c, zs);
                if (c != r) store_operand(e.next_fmt, ob, a.plane_elems, e.slab + (size_t)c * e.P + r, zs);
            }
        }
    } else {
        const float gl = gm[k1];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int c = c0 + j;
            if (c < e.n && r <= c) {
                const float gv = fmaf(gl, xn[j], g[j]);
                if (e.kind == CHAIN_FERMI && a.D) {
                    float dv;
                    if (e.flip) dv = (r == c ? (float)e.cdiag : 0.f) - gv;
                    else dv = gv + (r == c ? (float)e.cdiag : 0.f);
                    a.D[e.doff + (int64_t)r * e.n + c] = dv;
                    if (c != r) a.D[e.doff + (int64_t)c * e.n + r] = dv;
                }
                const double gd = (double)gv;
                if (r == c) {
                    tr += gd;
                    sq += gd * gd;
                } else {
                    sq += 2.0 * gd * gd;
                }
            }
        }
    }
}

// `scaled_in`: the products were formed from power-of-two scaled FP16 operands.
__device__ __forceinline__ void make_ctx(const LayerArgs& a, const Tile& t, int k, EpiCtx& e, bool scaled_in) {
    const ftsp2_instance in = a.inst[t.inst];
    const ftsp2_rescale_rec& rec = a.rec[t.inst];
    const DevModel& M = a.models[rec.model];
    e.n = in.n;
    e.P = a.P;
    e.chain = t.chain;
    e.kind = a.chain_kind[t.chain];
    e.flip = rec.flip;
    e.last = a.last;
    e.next_fmt = a.next_fmt;
    e.slab = (size_t)t.inst * a.P * a.P;
    e.doff = in.offset;
    e.L = a.layers[(e.kind == CHAIN_ENTROPY ? M.offS : M.off) + k];
    e.cdiag = rec.flip ? 1.0 - M.f0 : M.f0;
    e.mul = scaled_in ? e.L.acc_mul : e.L.a;
}

}  // namespace ftsp2
