// Internal declarations shared by the ftsp2 CUDA translation units.
//
// Centred recursion.  Every matrix chain is run in the variable
// Z_k = X_k - tau_k I, where tau_k is the image of the model's mu0 under the
// first k layers of the scalar recursion (tau_0 = mu0).  Substituting
// X_k = Z_k + tau_k I into Eq. mlsp2 gives, exactly,
//     Z_{k+1} = a_k Z_k^2 + (b_k + 2 a_k tau_k) Z_k           (no constant)
//     A_{k+1} = A_k + d_k Z_k          (the constant sum_k d_k tau_k moves
//                                         to the output)
//     D = A_L + Z_L + f0 I,  f0 = P_theta(mu0) = tau_L + sum_k d_k tau_k.
// The layer-0 state is Z_0 = H0 - mu0 I = scale (mu I - H) (Eq. H0 with the
// normalisation of Eqs. H', mu', beta' substituted; no division by the
// spectral width).  The products then only see deviations from the point
// where the Fermi function is steep, which keeps FP32 rounding far below the
// beta0/4 slope amplification that a plain X_k^2 suffers.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "ftsp2.h"

namespace ftsp2 {

constexpr int kMaxLayers = 64;
constexpr int kMaxMaxLayers = 20;            // Max-SP2 tables keep every layer: at most 20
int max_nparams(int L);                      // L (L + 5) / 2 + 2 numbers of a flat Max-SP2 table
constexpr int kMaxChains = 2;
constexpr int kTileM = 128;                  // tensor-core tile rows (UMMA M)
constexpr int kPad = 128;                    // matrix pitch granularity (elements)
constexpr int kPartialSlots = 32;            // FP64 partial-sum slots per tile (last layer)
constexpr int kEpiScratchFloats = 32768;     // deferred epilogue: finished sums of one CTA's tile
constexpr int kMaxDeferCtas = 192;           // CTAs with a scratch slot in the workspace
constexpr int kDeferMinK = 3072;             // default: deferred epilogue from this mean tile K
constexpr unsigned long long kDefaultWaitNs = 4000000000ull;   // 4 s: limit of a device-side wait

enum ChainKind : int { CHAIN_FERMI = 0, CHAIN_ENTROPY = 1 };

// Operand formats written for the next layer.
enum OpFmt : int { OP_F32 = 0, OP_TF32X3 = 1, OP_BF16X3 = 2, OP_F16X2 = 3 };

// Per layer constants of the centred recursion (float: what the epilogue uses).
// Per-layer constants of the centred epilogue.  From the product S = Z_k^2 and
// the stored state (Z_k, A):
//   xh = mul S + bp Z_k,   A' = A + d Z_k + d2 xh,   Z_{k+1} = p xh + q A,
// and at the last layer G = A + d Z_k + g xh.
// Eq. mlsp2: mul = a_k (times 2^(-2 e_k) for scaled FP16 products),
// bp = b_k + 2 a_k tau_k, d = d_k, d2 = 0, p = 1, q = 0, g = 1.
// Skip-SP2 (one stored layer, one accumulator; xh is the centred x_{k+1},
// A holds the centred A_{k+1}): mul = 2^(-2 e_k), bp = 2 sigma_k, d = 0,
// d2 = gamma_{k+1}, p = alpha_{k+1}, q = beta_{k+1}, and g = gamma_L.
struct DevLayer {
    float acc_mul;    // mul for scaled FP16 products (undoes 2^(2 e_k))
    float bp;
    float d;
    float out_scale;  // 2^(e_{k+1}): scale of the operands written for layer k+1
    float in_scale;   // 2^(e_k)
    float a;          // mul for unscaled products
    float p, q, d2, g;
    float pad0, pad1;
    // Max-SP2 layers (family FTSP2_FAMILY_MAX; FP32 mode): the layer reads the
    // nplanes stored centred layers x^_0 .. x^_{k} (state planes 0 .. k of the
    // chain) and its coefficients start at coef in the model set's pool:
    // theta_{k,0..k}, then theta_{k+1,0..k+1} (zeros after the last layer),
    // then, for the last layer, gamma_{0..L}.  nplanes = 0 for the other families.
    int coef, nplanes;
};

struct DevModel {
    double beta0, mu0, alpha;
    double f0;        // Fermi chain output at mu0
    double g0;        // entropy chain output at the centre mu0
    int L;            // Fermi chain layers
    int LS;           // entropy chain layers
    int off;          // first DevLayer of the Fermi chain (FP16 scales)
    int offS;         // first DevLayer of the entropy chain
    float scale0;     // 2^(e_0) of the Fermi chain (FP16 operands of Z_0)
    float scale0S;    // 2^(e_0) of the entropy chain
    // layer-0 state from the centred input X0 - mu0 I of each chain:
    // Z_0 = z0 (X0 - mu0 I), A = a0 (X0 - mu0 I) (Eq. mlsp2: 1, 0), and the
    // layer-0 operands op0 Z_0 (op0 = 1, except for Max-SP2, whose state plane
    // 0 holds x^_0 = X0 - mu0 I and whose operands are theta_00 x^_0)
    float z0, a0, z0S, a0S;
    float op0, op0S;
};

// One output tile of one grouped layer launch.
struct Tile {
    int inst;
    int I;            // BM-row block
    int J;            // BN-column block
    int chain;
};

// Per-instance bookkeeping written by the setup kernels (workspace).
struct InstWork {
    unsigned long long kmin, kmax;   // order-preserving keys of e_min / e_max
    int tile_start[2][kMaxChains];   // [tensor-core table, 128x128 table][chain]
    int tile_count[2][kMaxChains];
    int start_layer;                 // per chain, 16 bits each: first global layer
    int nonfinite;
};

struct Layout {
    // all offsets in bytes from the workspace base
    size_t inst_work, tiles, tiles_ref, partials, status, lanczos;
    size_t done;          // completion counters of multi-layer launches: kMaxLayers x nb x kMaxChains
    size_t escr;          // deferred-epilogue scratch (escr_ctas x kEpiScratchFloats floats)
    int escr_ctas;        // 0: the pair tiles run their final epilogue inline
    size_t Z[kMaxChains], A[kMaxChains], OP[kMaxChains][2], OPR[kMaxChains][2];
    size_t total;
    size_t plane_elems;   // nb * P * P
    int P, nb, nchains, ntiles, ntiles_ref, BN, BM;
    int planes;           // FP32 state planes per chain: 2 (Z, A), or L + 1 for Max-SP2 tables
};

// --- setup / bandwidth kernels (k_setup.cu) --------------------------------
struct SetupArgs {
    const double* H;
    const ftsp2_instance* inst;
    int nb, P, Lmax, nchains, BM, BN, BM_ref, BN_ref;
    const DevModel* models;
    int nmodels;
    int flags;
    int chain_kind[kMaxChains];
    InstWork* iw;
    Tile* tiles;
    Tile* tiles_ref;
    ftsp2_rescale_rec* rec;
    int* status;
    float* h32;                       // nullable: FP32 copy of H for FTSP2_LANCZOS, slab b at b P^2, row pitch P
    int* done;                        // per-instance completion counters, zeroed by prep
    int done_layers;                  // layers whose counters prep zeroes (done_layers x nb x kMaxChains)
};

void launch_prep(const SetupArgs& a, cudaStream_t s);
void launch_gershgorin(const SetupArgs& a, int max_n, cudaStream_t s);
void launch_decide(const SetupArgs& a, cudaStream_t s);

struct InitArgs {
    const double* H;
    const ftsp2_instance* inst;
    const ftsp2_rescale_rec* rec;
    const DevModel* models;
    const InstWork* iw;
    int nb, P, nchains;
    int chain_kind[kMaxChains];
    float* Z[kMaxChains];
    float* A[kMaxChains];
    uint8_t* OP[kMaxChains][2];    // operands in the main format
    uint8_t* OPR[kMaxChains][2];   // operands of refinement layers (nullable), format refine_fmt
    int main_fmt;                  // format of the main layers (OP_F32 in FTSP2_FP32 mode)
    int refine_fmt;                // OP_F32 (CUDA-core refinement) or OP_BF16X3 (FTSP2_REFINE_TC)
    int refine_from;               // global layers >= refine_from are refinement layers on OPR
    int upper_only;                // 16-bit operands as the upper triangle plus diagonal blocks
    size_t plane_elems;
};
void launch_init(const InitArgs& a, int max_n, cudaStream_t s);

struct FinalArgs {
    const ftsp2_instance* inst;
    ftsp2_rescale_rec* rec;
    const DevModel* models;
    const InstWork* iw;
    const double* partials;   // [tile][kPartialSlots][2]
    int table;                // tile table used by the last layer (0 main, 1 128x128)
    int nb, nchains;
    int chain_kind[kMaxChains];
    double* trace;            // nullable, [nb][2]
    double* S;                // nullable, [nb]
    const int* status;
};
void launch_finalize(const FinalArgs& a, cudaStream_t s);

// --- spectral bounds tightened by Lanczos (FTSP2_LANCZOS; k_lanczos.cu) ------------
constexpr int kLzSteps = 24;          // Lanczos steps (fewer when n is smaller)
constexpr int kLzRows = 8;            // matrix rows per block of the matvec (one warp each)
constexpr int kLzStopped = 0x10000;   // state flag: invariant subspace reached
struct LanczosArgs {
    const float* H32;                 // FP32 copy of H written by the Gershgorin pass (slab b at b P^2, pitch P)
    const ftsp2_instance* inst;
    InstWork* iw;                     // Gershgorin keys in, tightened keys out
    int nb, P, RB;                    // RB = ceil(P / kLzRows) partial sums per instance
    double* V0;                       // [nb][P] Lanczos vectors (ping-pong on the step parity)
    double* V1;
    double* W;                        // [nb][P] the next vector before normalisation
    float* V32;                       // [nb][P] FP32 copy of the current vector (matvec operand)
    double* ab;                       // [nb][kLzSteps][2] alpha_j, beta_j
    double* part;                     // [nb][RB]
    int* state;                       // [nb] steps done | kLzStopped
};
void launch_lanczos(const LanczosArgs& a, int max_n, int sms, cudaStream_t s);
// bytes of the Lanczos buffers for nb instances of pitch P (1024-aligned pieces)
size_t lanczos_ws_bytes(int nb, int P);
// carve the buffers out of ws (at least lanczos_ws_bytes(nb, P) bytes)
void lanczos_bind(LanczosArgs& a, uint8_t* ws, int nb, int P);

// --- chemical potential for a prescribed electron count (f1) ---------------------
struct MuArgs {
    ftsp2_instance* inst;            // device instance table; mu is updated in place
    const ftsp2_rescale_rec* rec;
    const double* trace;             // [nb][2]: Tr D, ||D||_F^2 at the current mu
    const double* nocc;              // [nb] prescribed electron counts
    int32_t* steps;                  // [nb] updates applied so far
    double tol;
    int nb;
};
void launch_mu_update(const MuArgs& a, cudaStream_t s);

// --- layer kernels -------------------------------------------------------------
struct LayerArgs {
    const Tile* tiles;
    int ntiles;
    const ftsp2_instance* inst;
    const ftsp2_rescale_rec* rec;
    const InstWork* iw;
    const DevModel* models;
    const DevLayer* layers;
    int P, Lmax, gl, last, nchains;
    int chain_kind[kMaxChains];
    int next_fmt;
    int chunk_elems;                  // K elements per TMEM accumulation chunk (0: kernel default)
    float* Z[kMaxChains];             // state (blocked layout); A[c] == Z[c] + plane_elems
    float* A[kMaxChains];
    const uint8_t* opr[kMaxChains];   // read operands (plane 0 base) - SIMT path
    uint8_t* opw[kMaxChains];         // write operands (plane 0 base)
    size_t plane_elems;
    float* D;
    double* partials;
    int* status;
    float* escr;                      // deferred final epilogue: kEpiScratchFloats per CTA, or null (inline)
    // Symmetric operands stored as the upper triangle plus the diagonal tile
    // blocks: lower_t = this layer's operands are stored so (K-slices left of
    // a panel's diagonal block are loaded transposed from the upper triangle);
    // mirror_all = this layer writes the mirror (c, r) everywhere (the next
    // layer reads full matrices), else only inside diagonal tiles.
    int lower_t, mirror_all;
    // Several consecutive layers in one persistent launch (nlayers > 1): the
    // work items are (global layer gl + l, tile) for l < nlayers, taken in that
    // order; an item of layer g waits until every epilogue of layer g - 1 of its
    // chain has finished (done[(g - 1) * kMaxChains + chain] reaches
    // kEpiWarps x CTAs per tile x tiles per chain).  Layers gl + 1, gl + 3, ...
    // write their operands through opw_alt and read them through the second
    // tensor-map set.  Layers >= tail_from accumulate chunk_tail elements per
    // TMEM chunk instead of chunk_elems.
    int nlayers;
    int chunk_tail, tail_from;
    uint8_t* opw_alt[kMaxChains];
    // completion counters of multi-layer launches, one per (layer, instance,
    // chain): done_inst[(g * nb + instance) * kMaxChains + chain]; an item waits
    // for its own instance's previous layer
    int* done_inst;
    int nb;
    int dtab;                         // tile table of this launch in InstWork (0 main, 1 128 x 128)
    // Time limit of one device-side wait (ns; ftsp2_set_wait_limit_ns).  A
    // dependency wait that runs out records FTSP2_E_TIMEOUT and the launch
    // finishes its work list in skip mode; a pipeline wait records it after
    // wait_ns and gives up after 2 wait_ns.
    const float* coef;                // Max-SP2 coefficient pool of the model set (nullable)
    unsigned long long wait_ns;
    // Test hook (ftsp2_debug_stall_layer): items of this global layer wait for
    // one completion more than their predecessor layer can give, so that the
    // dependency wait runs out; -1 in normal operation.
    int stall_layer;
};

struct TmaMaps {
    CUtensorMap a[kMaxChains][3];   // [chain][split plane], boxes of 128 rows x 128 bytes
    CUtensorMap t[kMaxChains][3];   // 16-bit planes: boxes of 64 rows x 64 columns (transposed panels)
};

// Tensor-core layer (k_layer_tc.cu); mode in {TF32X3, BF16X3, FP16X2}.
int tc_block_n(int mode, int pair);
int tc_block_m(int mode, int pair);
int tc_smem_bytes(int mode);
// pair = 1: 256 x 256 tiles on CTA pairs (units = pairs); pair = 0: 128 x 128
// tiles on single CTAs (units = CTAs).  Persistent grid of `units`.
cudaError_t launch_layer_tc(int mode, const LayerArgs& a, const TmaMaps& maps, const TmaMaps& maps_alt, int units,
                            int pair, cudaStream_t s);
// Largest number of units (pairs or CTAs) of the main-format layer kernel that
// can be resident at once (0 if unknown): the bound for multi-layer launches,
// whose CTAs wait on one another.
int layer_tc_max_units(int mode, int pair, bool defer);
// CUDA-core FP32 layer (k_layer_simt.cu), 128 x 128 tiles.
cudaError_t launch_layer_simt(const LayerArgs& a, int grid, cudaStream_t s);

// --- training (k_train.cu) -----------------------------------------------------
struct ThetaParam {
    double v[4 * kMaxLayers];
};
// family FTSP2_FAMILY_MLSP2: th = L rows (a, b, c, d), 4L Jacobian columns;
// FTSP2_FAMILY_SKIP: th = L rows (delta, alpha, beta, gamma) + (A_0, gamma_L),
// 4L + 2 columns; FTSP2_FAMILY_MAX: th = the flat Max-SP2 table, L (L + 5) / 2
// + 2 columns (L <= 20: at most 252 entries).  The residual column follows the
// Jacobian's.
cudaError_t launch_train_fwd_jac(int target, double beta0, double mu0, int L, double alpha,
                                 const ThetaParam& th, const double* dX, int ns,
                                 double* dR, double* dM, cudaStream_t s, int family = FTSP2_FAMILY_MLSP2);
cudaError_t launch_train_residual(int target, double beta0, double mu0, int L, double alpha,
                                  const ThetaParam& th, const double* dX, int ns,
                                  double* dR, cudaStream_t s, int family = FTSP2_FAMILY_MLSP2);
cudaError_t launch_train_gram(const double* dM, int ns, int np, double* dG, double* dScratch,
                              int nchunks, cudaStream_t s);
cudaError_t launch_train_accel(const double* dM, const double* dV, const double* dRh, double h,
                               int ns, int np, double* dPart, double* dOut, cudaStream_t s);
cudaError_t launch_train_absmax(const double* dR, int ns, double* dPart, double* dOut,
                                cudaStream_t s);

void count_launch(int n = 1);

// --- inputs of the training built by the library (train_inputs.cu, host) ----------
// N sample points of [0, 1] at the quantiles of p = 1 + |f'| (seed 0: cell
// midpoints; else splitmix64-drawn positions inside the N cells)
void train_sample_grid(double beta0, double mu0, int N, uint64_t seed, double* x);
// starting tables: the SP2-mu sequence at mu0 with the slope-matching
// contraction in layer 0 (L rows of 4), the same sequence in the one-term form
// (L + 1 rows of 2), and the Appendix embedding of Eq. mlsp2 rows in Skip-SP2
// (L + 1 rows of 4)
void train_init_mlsp2(int L, double beta0, double mu0, double* theta);
void train_init_alt(int L, double mu0, double* alt);
void mlsp2_to_skip(int L, const double* theta, double* tab);

// Element offset of (r, c) inside one P x P slab of the FP32 state Z, A (P a
// multiple of 128).  The slab is cut into blocks of 32 rows x 8 columns (1 KB),
// stored block row by block row; a block holds two 32 x 4 halves, each with the
// 4 columns of a row contiguous.  An epilogue warp whose lane i owns row
// r0 + i (r0 % 32 == 0) reads 4 consecutive columns (c % 4 == 0) of its 32 rows
// as one contiguous 512-byte run, and the 32 x W region of a warp is W / 8
// consecutive blocks.  Only the layer epilogues and the initialisation touch
// the state, so its layout is free of the operands' row-major constraint.
__host__ __device__ __forceinline__ size_t state_off(int P, int r, int c) {
    return ((size_t)(r >> 5) * (size_t)(P >> 3) + (size_t)(c >> 3)) * 256 + (size_t)(((c >> 2) & 1) * 128) +
           (size_t)((r & 31) * 4 + (c & 3));
}

}  // namespace ftsp2

// ---------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace ftsp2 {

__device__ __forceinline__ unsigned long long dkey(double x) {
    // order-preserving map of doubles onto unsigned 64-bit integers
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dunkey(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

}  // namespace ftsp2
#endif
