// C ABI of the ftsp2 library: model sets, workspace planning, the launch
// sequence of the hot path, and the Levenberg-Marquardt driver of the
// training path.  Host code only; kernels live in k_*.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ftsp2_internal.h"

namespace ftsp2 {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// event pairs around tensor-core layer launches (measurement support)
static std::mutex g_prof_mu;
static bool g_prof_on = false;
struct ProfEvent {
    cudaEvent_t e0, e1;
    int layers;
};
static std::vector<ProfEvent> g_prof_events;
// multi-layer (cooperative) launches: 1 usable, 0 refused once, -1 not tried
static std::atomic<int> g_coop_ok{-1};
// limit of each bounded device-side wait, and the dependency-stall test hook
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};
static std::atomic<int> g_stall_layer{-1};

// ------------------------------------------------------------------------------
// device checks and the CUDA driver API's tensor-map encoder
// ------------------------------------------------------------------------------
struct DeviceInfo {
    int sms = 0;
    int major = 0, minor = 0;
};

static ftsp2_status device_info(DeviceInfo& di) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FTSP2_E_CUDA;
    static std::mutex mu;
    static int cached_dev = -1;
    static DeviceInfo cached;
    std::lock_guard<std::mutex> lk(mu);
    if (cached_dev != dev) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return FTSP2_E_CUDA;
        cached.sms = p.multiProcessorCount;
        cached.major = p.major;
        cached.minor = p.minor;
        cached_dev = dev;
    }
    di = cached;
    if (di.major != 10 || di.minor != 3) return FTSP2_E_UNSUPPORTED;
    return FTSP2_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map over a stack of nb padded P x P slabs (rows = nb * P), element type
// `dt`, box {box_k elements, box_rows rows}, 128-byte swizzle.
static bool encode_map(CUtensorMap* m, void* base, CUtensorMapDataType dt, int esize, int P, int nb, int box_k,
                       int box_rows) {
    auto fn = encoder();
    if (!fn) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)P, (cuuint64_t)nb * (cuuint64_t)P};
    cuuint64_t gstride[1] = {(cuuint64_t)P * (cuuint64_t)esize};
    cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, dt, 2, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------------------
// model sets
// ------------------------------------------------------------------------------
struct HostModel {
    int L = 0, LS = 0;
    int family = FTSP2_FAMILY_MLSP2;
    double beta0 = 0, mu0 = 0, alpha = 0;
    std::vector<double> th, thS;   // Eq. mlsp2: 4L; Skip-SP2: 4(L + 1) (output row last)
};

}  // namespace ftsp2

struct ftsp2_model_set {
    std::vector<ftsp2::HostModel> host;
    ftsp2::DevModel* d_models[2] = {nullptr, nullptr};   // [plain, fp16-scaled]
    ftsp2::DevLayer* d_layers[2] = {nullptr, nullptr};
    void* d_mem = nullptr;
    float* d_coef = nullptr;       // Max-SP2 coefficient pool (nullable)
    int Lmax = 0;
    int planes = 2;                // FP32 state planes per chain a solve needs
    bool has_max = false;
    int device = -1;
};

namespace ftsp2 {

// FP16 range control: 2^e with 1.25 max|Z| 2^e <= 2^14 (0 when unscaled).
static int fp16_exponent(double m, bool scaled) {
    if (!scaled || !(m > 0.0)) return 0;
    const int ek = (int)std::floor(std::log2(16384.0 / (1.25 * m)));
    return std::min(40, std::max(-20, ek));
}

// Skip-SP2 chain (one stored layer, one accumulator): the centre trajectory at
// x0 = mu0 (sigma_k of the squared combination, chi_k of x_k, rho_k of A_k),
// the FP16 exponents from max over the inputs of |u_k - sigma_k|, and the
// epilogue constants of DevLayer.
static void chain_constants_skip(const std::vector<double>& tb, int L, double mu0, double lo, double hi,
                                 bool scaled, std::vector<DevLayer>& out, double& f0, float& scale0, float& z0,
                                 float& a0) {
    std::vector<double> sig(L), chi(L + 1), rho(L + 1);
    chi[0] = mu0;
    rho[0] = tb[4 * L];
    for (int k = 0; k < L; ++k) {
        const double dl = tb[4 * k], al = tb[4 * k + 1], be = tb[4 * k + 2], ga = tb[4 * k + 3];
        sig[k] = dl + al * chi[k] + be * rho[k];
        rho[k + 1] = rho[k] + ga * chi[k];
        chi[k + 1] = sig[k] * sig[k];
    }
    const double gL = tb[4 * L + 1];
    f0 = rho[L] + gL * chi[L];
    const int G = 20001;
    std::vector<double> x(G), A(G, tb[4 * L]);
    for (int i = 0; i < G; ++i) x[i] = lo + (hi - lo) * (double)i / (G - 1);
    std::vector<int> e(L + 1, 0);
    for (int k = 0; k < L; ++k) {
        const double dl = tb[4 * k], al = tb[4 * k + 1], be = tb[4 * k + 2], ga = tb[4 * k + 3];
        double m = 0.0;
        for (int i = 0; i < G; ++i) {
            const double u = dl + al * x[i] + be * A[i];
            m = std::max(m, std::fabs(u - sig[k]));
            A[i] += ga * x[i];
            x[i] = u * u;
        }
        e[k] = fp16_exponent(m, scaled);
    }
    out.resize(L);
    for (int k = 0; k < L; ++k) {
        DevLayer dl;
        dl.a = 1.f;
        dl.acc_mul = (float)std::ldexp(1.0, -2 * e[k]);
        dl.bp = (float)(2.0 * sig[k]);
        dl.d = 0.f;
        dl.in_scale = (float)std::ldexp(1.0, e[k]);
        if (k + 1 < L) {
            dl.p = (float)tb[4 * (k + 1) + 1];
            dl.q = (float)tb[4 * (k + 1) + 2];
            dl.d2 = (float)tb[4 * (k + 1) + 3];
            dl.g = 0.f;
            dl.out_scale = (float)std::ldexp(1.0, e[k + 1]);
        } else {
            dl.p = dl.q = dl.d2 = 0.f;
            dl.g = (float)gL;
            dl.out_scale = 1.f;
        }
        dl.pad0 = dl.pad1 = 0.f;
        dl.coef = -1;
        dl.nplanes = 0;
        out[k] = dl;
    }
    scale0 = (float)std::ldexp(1.0, e[0]);
    z0 = (float)tb[1];
    a0 = (float)tb[3];
}

// Trajectory of the centre and the per-layer constants of one chain.
// x0range: interval of layer-0 inputs the chain sees (subset of [0, 1]).
static void chain_constants(const std::vector<double>& th, int L, double mu0, double lo, double hi, bool scaled,
                            std::vector<DevLayer>& out, double& f0, float& scale0) {
    std::vector<double> tau(L + 1);
    tau[0] = mu0;
    for (int k = 0; k < L; ++k) {
        const double a = th[4 * k], b = th[4 * k + 1], c = th[4 * k + 2];
        tau[k + 1] = a * tau[k] * tau[k] + b * tau[k] + c;
    }
    f0 = tau[L];
    for (int k = 0; k < L; ++k) f0 += th[4 * k + 3] * tau[k];
    // spectral radius bound of the centred state: max over inputs of |x_k - tau_k|
    const int G = 20001;
    std::vector<double> x(G);
    for (int i = 0; i < G; ++i) x[i] = lo + (hi - lo) * (double)i / (G - 1);
    std::vector<int> e(L + 1, 0);
    for (int k = 0; k <= L; ++k) {
        double m = 0.0;
        for (int i = 0; i < G; ++i) m = std::max(m, std::fabs(x[i] - tau[k]));
        if (scaled && m > 0.0) {
            int ek = (int)std::floor(std::log2(16384.0 / (1.25 * m)));
            e[k] = std::min(40, std::max(-20, ek));
        }
        if (k < L) {
            const double a = th[4 * k], b = th[4 * k + 1], c = th[4 * k + 2];
            for (int i = 0; i < G; ++i) x[i] = a * x[i] * x[i] + b * x[i] + c;
        }
    }
    out.resize(L);
    for (int k = 0; k < L; ++k) {
        const double a = th[4 * k], b = th[4 * k + 1], d = th[4 * k + 3];
        DevLayer dl;
        dl.a = (float)a;
        dl.acc_mul = (float)(a * std::ldexp(1.0, -2 * e[k]));
        dl.bp = (float)(b + 2.0 * a * tau[k]);
        dl.d = (float)d;
        dl.in_scale = (float)std::ldexp(1.0, e[k]);
        dl.out_scale = (float)std::ldexp(1.0, e[k + 1]);
        dl.p = 1.f;
        dl.q = 0.f;
        dl.d2 = 0.f;
        dl.g = 1.f;
        dl.pad0 = dl.pad1 = 0.f;
        dl.coef = -1;
        dl.nplanes = 0;
        out[k] = dl;
    }
    scale0 = (float)std::ldexp(1.0, e[0]);
}

// Max-SP2 chain (FTSP2_FAMILY_MAX, FP32 mode): the centre trajectory at
// x0 = mu0 (chi_j of x_j, sigma_i of u_i), f0 = c + sum_j gamma_j chi_j, and per
// layer the coefficient block of the pool (DevLayer.coef): theta_{i,0..i},
// theta_{i+1,0..i+1} (zeros after the last layer), and gamma_{0..L} for the
// last layer.  In the centred variables x^_j = x_j - chi_j the layer i computes
// Z^_i = sum_j theta_{i,j} x^_j, x^_{i+1} = S + 2 sigma_i Z^_i (S = Z^_i^2), and
// Z^_{i+1} = sum_{j <= i+1} theta_{i+1,j} x^_j (the constants cancel).
int max_nparams(int L) { return L * (L + 5) / 2 + 2; }
static void chain_constants_max(const std::vector<double>& p, int L, double mu0, std::vector<DevLayer>& out,
                                std::vector<float>& pool, double& f0, float& op0) {
    std::vector<int> off(L);
    int o = 0;
    for (int i = 0; i < L; ++i) {
        off[i] = o;
        o += i + 3;
    }
    const double c = p[o], gL = p[o + 1];
    auto theta = [&](int i, int j) { return p[off[i] + 2 + j]; };
    auto gamma = [&](int j) { return j < L ? p[off[j] + 1] : gL; };
    std::vector<double> chi(L + 1), sig(L);
    chi[0] = mu0;
    for (int i = 0; i < L; ++i) {
        double u = p[off[i]];
        for (int j = 0; j <= i; ++j) u += theta(i, j) * chi[j];
        sig[i] = u;
        chi[i + 1] = u * u;
    }
    f0 = c;
    for (int j = 0; j <= L; ++j) f0 += gamma(j) * chi[j];
    out.resize(L);
    for (int i = 0; i < L; ++i) {
        DevLayer dl;
        std::memset(&dl, 0, sizeof(dl));
        dl.a = dl.acc_mul = 1.f;
        dl.bp = (float)(2.0 * sig[i]);
        dl.in_scale = dl.out_scale = 1.f;
        dl.coef = (int)pool.size();
        dl.nplanes = i + 1;
        for (int j = 0; j <= i; ++j) pool.push_back((float)theta(i, j));
        for (int j = 0; j <= i + 1; ++j) pool.push_back(i + 1 < L ? (float)theta(i + 1, j) : 0.f);
        if (i == L - 1)
            for (int j = 0; j <= L; ++j) pool.push_back((float)gamma(j));
        out[i] = dl;
    }
    op0 = (float)theta(0, 0);
}

static ftsp2_status upload_models(ftsp2_model_set* s) {
    const int nm = (int)s->host.size();
    std::vector<DevModel> dm[2];
    std::vector<DevLayer> dl[2];
    std::vector<float> pool[2];
    for (int v = 0; v < 2; ++v) {
        const bool scaled = v == 1;
        for (int m = 0; m < nm; ++m) {
            const HostModel& h = s->host[m];
            DevModel M;
            M.beta0 = h.beta0;
            M.mu0 = h.mu0;
            M.alpha = h.alpha;
            M.L = h.L;
            M.LS = h.LS;
            std::vector<DevLayer> lf, ls;
            const double ylo = h.mu0 + h.alpha * (0.0 - h.mu0), yhi = h.mu0 + h.alpha * (1.0 - h.mu0);
            const std::vector<double>& thE = h.thS.empty() ? h.th : h.thS;
            if (h.family == FTSP2_FAMILY_MAX) {
                // FP32 mode only: no FP16 scales; state plane 0 = x^_0 (z0 = 1)
                chain_constants_max(h.th, h.L, h.mu0, lf, pool[v], M.f0, M.op0);
                chain_constants_max(thE, h.LS, h.mu0, ls, pool[v], M.g0, M.op0S);
                M.scale0 = M.scale0S = 1.f;
                M.z0 = M.z0S = 1.f;
                M.a0 = M.a0S = 0.f;
            } else if (h.family == FTSP2_FAMILY_SKIP) {
                chain_constants_skip(h.th, h.L, h.mu0, 0.0, 1.0, scaled, lf, M.f0, M.scale0, M.z0, M.a0);
                chain_constants_skip(thE, h.LS, h.mu0, std::min(ylo, yhi), std::max(ylo, yhi), scaled, ls, M.g0,
                                     M.scale0S, M.z0S, M.a0S);
                M.op0 = M.op0S = 1.f;
            } else {
                chain_constants(h.th, h.L, h.mu0, 0.0, 1.0, scaled, lf, M.f0, M.scale0);
                chain_constants(thE, h.LS, h.mu0, std::min(ylo, yhi), std::max(ylo, yhi), scaled, ls, M.g0,
                                M.scale0S);
                M.z0 = M.z0S = 1.f;
                M.a0 = M.a0S = 0.f;
                M.op0 = M.op0S = 1.f;
            }
            M.off = (int)dl[v].size();
            dl[v].insert(dl[v].end(), lf.begin(), lf.end());
            M.offS = (int)dl[v].size();
            dl[v].insert(dl[v].end(), ls.begin(), ls.end());
            dm[v].push_back(M);
        }
    }
    const size_t bm = sizeof(DevModel) * nm, bl = sizeof(DevLayer) * dl[0].size();
    const size_t bp = (sizeof(float) * pool[0].size() + 255) / 256 * 256;
    const size_t bm_a = (bm + 255) / 256 * 256, bl_a = (bl + 255) / 256 * 256;
    const size_t total = 2 * (bm_a + bl_a) + bp + 256;
    if (cudaMalloc(&s->d_mem, total) != cudaSuccess) return FTSP2_E_CUDA;
    uint8_t* p = static_cast<uint8_t*>(s->d_mem);
    for (int v = 0; v < 2; ++v) {
        s->d_models[v] = reinterpret_cast<DevModel*>(p);
        p += bm_a;
        s->d_layers[v] = reinterpret_cast<DevLayer*>(p);
        p += bl_a;
        if (cudaMemcpy(s->d_models[v], dm[v].data(), bm, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->d_layers[v], dl[v].data(), bl, cudaMemcpyHostToDevice) != cudaSuccess)
            return FTSP2_E_CUDA;
    }
    // the Max-SP2 coefficient pool (FP32 mode uses the unscaled variant)
    s->d_coef = nullptr;
    if (!pool[0].empty()) {
        s->d_coef = reinterpret_cast<float*>(p);
        if (cudaMemcpy(s->d_coef, pool[0].data(), sizeof(float) * pool[0].size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return FTSP2_E_CUDA;
    }
    cudaGetDevice(&s->device);
    return FTSP2_OK;
}

// Table printed in the paper's Appendix A (beta0 = 1500, mu0 = 1/3):
// rows (a, b, c, d) of Eq. mlsp2.
static const double kPrinted[26][4] = {
    {-1.353996666080607e+00, +2.437540893737664e+00, -2.038466804171965e-01, +1.291156147536192e-11},
    {+1.608677030263155e+00, -2.987544634415441e-01, -6.746741346599809e-02, -7.006084032292678e-12},
    {-2.351636735892118e+00, +2.613813908880740e+00, -2.081115324436639e-03, -6.572840812953572e-13},
    {+1.810031371507046e+00, -3.733036049410451e-02, -5.442179841399564e-02, +4.318503541775794e-11},
    {-2.732204264661287e+00, +2.825886342002125e+00, +8.167975559885774e-03, -1.662456055798004e-11},
    {-1.873987421378235e+00, +2.138798318408699e+00, +3.573114610928145e-02, +4.542623791264443e-12},
    {+1.402261079424850e+00, +4.890736627204146e-02, -4.237220339751432e-02, +2.424648524635838e-11},
    {+1.713089400763156e+00, -1.034037621506357e-01, -2.438094942357169e-02, +7.873381643056254e-11},
    {-3.252595736449542e+00, +2.628649626717414e+00, +3.165347918592593e-02, -6.312379678783267e-11},
    {-1.878046620274372e+00, +2.074880349608742e+00, +3.449163838903798e-02, -6.649574392039178e-11},
    {+1.310464008049612e+00, +5.496499701340592e-02, +3.310087064751345e-03, +2.825980776677432e-10},
    {+1.563608995897714e+00, -8.606990671650539e-03, -1.301065468049911e-02, -1.424083924407828e-07},
    {-3.038983738437103e+00, +2.477686862799397e+00, +2.636871201950337e-02, -1.330100571490071e-07},
    {-1.699377329573085e+00, +2.076565284757246e+00, +3.442469802192470e-02, +4.896446563691430e-03},
    {+1.256940670391469e+00, +5.777573303514125e-02, +4.902596975631270e-02, -2.302054912581413e-03},
    {-1.390281989291434e+00, +1.966243706278270e+00, +1.910503489826946e-02, +1.606259300834474e-02},
    {+1.172415492052006e+00, +2.982302801604828e-02, +4.530045685625948e-02, -1.539021333689731e-02},
    {+1.351448045975672e+00, +5.773064380022182e-02, +3.753306163777001e-02, -1.276795931125504e-01},
    {-1.212734900653146e+00, +1.861660915086903e+00, +1.242573869144004e-02, -1.100276149057915e-01},
    {+8.610663421144649e-01, +1.048747203546148e-02, +4.701135000272372e-02, -4.946843804326570e-02},
    {-1.369173339062334e+00, +1.699077704335121e+00, -7.732969926664974e-03, -1.761228530611925e-01},
    {-1.452079661340262e+00, +1.993171071701545e+00, -1.661115887219701e-02, -5.688902388963853e-01},
    {+1.347262922911275e+00, +2.198074427424086e-02, +1.995615256168758e-01, +5.964487309001580e-01},
    {-1.114238353358810e+00, +1.896937623313116e+00, -7.280733281872145e-02, +1.530915295291056e+00},
    {+9.411010738180853e-01, -1.554719335561439e-01, +6.584253835393120e-02, -2.059339861429303e-01},
    {+8.321693583250559e-01, +5.698259888759222e-01, -4.234806053199446e-01, +5.698259888760550e-01},
};

// ------------------------------------------------------------------------------
// workspace planning
// ------------------------------------------------------------------------------
static int fmt_of_mode(int mode) {
    switch (mode) {
        case FTSP2_FP16X2: return OP_F16X2;
        case FTSP2_BF16X3: return OP_BF16X3;
        case FTSP2_TF32X3: return OP_TF32X3;
        default: return OP_F32;
    }
}
static int op_bytes(int fmt) {
    switch (fmt) {
        case OP_F16X2: return 4;
        case OP_BF16X3: return 6;
        case OP_TF32X3: return 8;
        default: return 4;
    }
}
// K elements per TMEM accumulation chunk of a tensor-core layer.  FP16X2:
// 128, and 64 for the last kShortChunkLayers layers; BF16X3 and TF32X3, whose
// layers carry more MMA work per drained chunk (6 products, or half-rate TF32),
// so that shorter chunks cost almost nothing: 64 for every layer.  Measured at
// n = 2048 (8x16x16 lattice, printed table, density + entropy; n = 4096 alike),
// max|D - D_ref| / |S - S_ref|/n:
//   FP16X2 128 + last 6 at 64:  1.00e-6 / 8.9e-7  (n = 2048)
//   FP16X2 128 + last 12 at 64: 7.6e-7 / 6.2e-7, +2 to 3 % time
//   BF16X3 128 + last 6 at 64:  8.3e-7 / 1.08e-6;  64 everywhere: 5.0e-7 / 8.0e-7, +0.2 %
//   TF32X3 128 + last 6 at 64:  9.7e-7 / 1.25e-6;  64 everywhere: 6.2e-7 / 8.3e-7, +0.6 %
// Batches of short tiles (mean order n over the launch's tiles below
// kShortTileK, e.g. ragged batches of n <= 768) run 64-element chunks in every
// layer: their tiles carry little MMA work against the epilogue's memory
// traffic, so the extra chunk drains cost almost nothing, and the rounding of
// the high-beta0 models such batches select stays smaller.
constexpr int kShortChunkLayers = 12;
constexpr double kShortTileK = 1024.0;
static int chunk_elems_of(int mode, int g, int Lmax, double mean_k) {
    if (mode == FTSP2_BF16X3 || mode == FTSP2_TF32X3) return 64;
    if (mean_k < kShortTileK) return 64;
    return g >= Lmax - kShortChunkLayers ? 64 : 0;    // 0: the kernel's default (128)
}

static int refine_layers(int flags) { return (flags & FTSP2_REFINE2) ? 2 : ((flags & FTSP2_REFINE1) ? 1 : 0); }

static int host_tiles_of(int n, int BM, int BN) {
    const int q = BN / BM;
    const int nI = (n + BM - 1) / BM;
    const int nJ = (n + BN - 1) / BN;
    int c = 0;
    for (int J = 0; J < nJ; ++J) c += std::min(q * (J + 1), nI);
    return c;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static ftsp2_status plan(const ftsp2_instance* inst, int nb, int mode, int want, int flags, Layout& L,
                         int planes = 2) {
    if (!inst || nb < 1) return FTSP2_E_ARG;
    if (mode < FTSP2_FP32 || mode > FTSP2_FP16X2) return FTSP2_E_ARG;
    if (want < 1 || want > 3) return FTSP2_E_ARG;
    int maxn = 0;
    for (int b = 0; b < nb; ++b) {
        if (inst[b].n < 1 || inst[b].offset < 0) return FTSP2_E_ARG;
        maxn = std::max(maxn, inst[b].n);
    }
    const int P = (int)align_up((size_t)maxn, kPad);
    const int nch = want == 3 ? 2 : 1;
    const bool simt_main = mode == FTSP2_FP32;
    // main tile table: 256 x 256 pair tiles (tensor-core modes) or 128 x 128
    // (FP32 mode); the 128 x 128 table serves single-CTA tensor-core layers and
    // FP32 refinement layers
    const int BN = simt_main ? 128 : tc_block_n(mode, 1);
    const int BM = simt_main ? 128 : tc_block_m(mode, 1);
    const bool refine = !simt_main && refine_layers(flags) > 0;
    const bool need_ref = !simt_main;
    long long nt = 0, ntr = 0;
    double tile_k = 0.0;                       // sum of the orders n over the pair tiles
    for (int b = 0; b < nb; ++b) {
        const long long t = host_tiles_of(inst[b].n, BM, BN);
        nt += t;
        tile_k += (double)t * inst[b].n;
        if (need_ref) ntr += host_tiles_of(inst[b].n, 128, 128);
    }
    // deferred final epilogue of the pair tiles: by default when their mean
    // K is long enough for two store warps to keep up with the MMAs
    const bool defer = !simt_main && !(flags & FTSP2_EPI_INLINE) &&
                       ((flags & FTSP2_EPI_DEFERRED) || tile_k >= (double)kDeferMinK * (double)nt);
    nt *= nch;
    ntr *= nch;
    if (nt > (1ll << 30)) return FTSP2_E_ARG;
    L.P = P;
    L.nb = nb;
    L.nchains = nch;
    L.ntiles = (int)nt;
    L.ntiles_ref = (int)ntr;
    L.BN = BN;
    L.BM = BM;
    L.plane_elems = (size_t)nb * P * P;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 1024);
        return o;
    };
    L.status = take(256);
    L.done = take(sizeof(int) * kMaxLayers * kMaxChains * (size_t)nb);
    L.inst_work = take(sizeof(InstWork) * nb);
    L.tiles = take(sizeof(Tile) * nt);
    L.tiles_ref = need_ref ? take(sizeof(Tile) * ntr) : 0;
    L.partials = take(sizeof(double) * 2 * kPartialSlots * std::max<long long>(nt, ntr));
    L.lanczos = take(lanczos_ws_bytes(nb, P));   // used with FTSP2_LANCZOS only
    L.escr_ctas = defer ? (int)std::min<long long>(kMaxDeferCtas, 2 * nt) : 0;
    L.escr = L.escr_ctas ? take((size_t)L.escr_ctas * kEpiScratchFloats * sizeof(float)) : 0;
    const int fmt = fmt_of_mode(mode);
    for (int c = 0; c < kMaxChains; ++c) {
        L.Z[c] = L.A[c] = L.OP[c][0] = L.OP[c][1] = L.OPR[c][0] = L.OPR[c][1] = 0;
    }
    L.planes = std::max(2, planes);
    for (int c = 0; c < nch; ++c) {
        // state planes 0 .. planes - 1 back to back: Z, A, then the further
        // stored layers of Max-SP2 tables (plane j at Z + j plane_elems)
        L.Z[c] = take(4 * L.plane_elems * (size_t)L.planes);
        L.A[c] = L.Z[c] + 4 * L.plane_elems;
        L.OP[c][0] = take((size_t)op_bytes(fmt) * L.plane_elems);
        L.OP[c][1] = take((size_t)op_bytes(fmt) * L.plane_elems);
        if (refine) {
            const size_t rb = (flags & FTSP2_REFINE_TC) ? (size_t)op_bytes(OP_BF16X3) : 4;
            L.OPR[c][0] = take(rb * L.plane_elems);
            L.OPR[c][1] = take(rb * L.plane_elems);
        }
    }
    // the layer epilogues address A_c as Z_c + plane_elems
    for (int c = 0; c < nch; ++c)
        if (L.A[c] != L.Z[c] + 4 * L.plane_elems) return FTSP2_E_WORKSPACE;
    L.total = off;
    return FTSP2_OK;
}

static ftsp2_status from_cuda(cudaError_t e) { return e == cudaSuccess ? FTSP2_OK : FTSP2_E_CUDA; }

// ---- tile-shape choice (autotuner) --------------------------------------------
// Tensor-core layers run either on CTA pairs with 256 x 256 tiles or on single
// CTAs with 128 x 128 tiles.  The choice is per batch signature (device, mode,
// chains, refinement, the sorted list of orders n): ftsp2_autotune measures both
// and records the faster; otherwise a padding model decides.
static std::mutex g_tune_mu;
static std::map<uint64_t, int> g_tune;

static uint64_t batch_signature(const ftsp2_instance* inst, int nb, int mode, int want, int flags) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int> ns(nb);
    for (int b = 0; b < nb; ++b) ns[b] = inst[b].n;
    std::sort(ns.begin(), ns.end());
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix((uint64_t)dev);
    mix((uint64_t)mode);
    mix((uint64_t)want);
    mix((uint64_t)refine_layers(flags));
    mix((uint64_t)nb);
    for (int v : ns) mix((uint64_t)v);
    return h;
}

// Padding model: multiply-adds issued per layer (tiles x tile^2 x n) divided by
// the number of units that run them in parallel, with the waves rounded up.
static int shape_by_model(const ftsp2_instance* inst, int nb, int sms) {
    double cost[2] = {0.0, 0.0};
    for (int pair = 0; pair < 2; ++pair) {
        const int T = pair ? 256 : 128;
        const int units = pair ? sms / 2 : sms;
        double work = 0.0;
        long long tiles = 0;
        for (int b = 0; b < nb; ++b) {
            const long long t = host_tiles_of(inst[b].n, T, T);
            tiles += t;
            work += (double)t * T * T * inst[b].n;
        }
        const double waves = std::ceil((double)tiles / std::max(1, units));
        const double per_tile = work / std::max<long long>(1, tiles);
        // a pair tile moves half of B per SM; count its MMA work at 0.8
        cost[pair] = waves * per_tile / (pair ? 2.0 : 1.0) * (pair ? 0.8 : 1.0);
    }
    return cost[1] <= cost[0] ? 1 : 0;
}

static int tile_shape_choice(const ftsp2_instance* inst, int nb, int mode, int want, int flags, int sms,
                             int* from_tuner = nullptr) {
    if (from_tuner) *from_tuner = 0;
    if (flags & FTSP2_PAIR_TILES) return 1;
    if (flags & FTSP2_SINGLE_TILES) return 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(batch_signature(inst, nb, mode, want, flags));
        if (it != g_tune.end()) {
            if (from_tuner) *from_tuner = 1;
            return it->second;
        }
    }
    return shape_by_model(inst, nb, sms);
}

// The launch sequence of (a1)-(a6).
static ftsp2_status run(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst, int nb,
                        const ftsp2_model_set* set, int mode, int flags, int want, float* dD, double* dTrace,
                        double* dS, ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes, void* stream) {
    if (!set || set->host.empty()) return FTSP2_E_NOMODEL;
    if (!dH || !dInst || !dRec || !ws) return FTSP2_E_ARG;
    if ((want & 1) && !dD && !dTrace) return FTSP2_E_ARG;
    if ((want & 2) && !dS) return FTSP2_E_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % 1024 != 0) return FTSP2_E_WORKSPACE;
    DeviceInfo di;
    ftsp2_status st = device_info(di);
    if (st != FTSP2_OK) return st;
    // Max-SP2 tables keep every layer: FP32 mode (CUDA-core layers) only
    if (set->has_max && mode != FTSP2_FP32) return FTSP2_E_UNSUPPORTED;
    Layout L;
    st = plan(inst, nb, mode, want, flags, L, set->planes);
    if (st != FTSP2_OK) return st;
    if (ws_bytes < L.total) return FTSP2_E_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // launches on a stream being captured into a CUDA graph are recorded, not
    // run: no synchronising, and the layer profiling events stay off
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return FTSP2_E_CUDA;
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (capturing && (flags & FTSP2_SYNC)) return FTSP2_E_ARG;
    uint8_t* W = static_cast<uint8_t*>(ws);
    const bool scaled = mode == FTSP2_FP16X2;
    const DevModel* models = set->d_models[scaled ? 1 : 0];
    const DevLayer* layers = set->d_layers[scaled ? 1 : 0];
    const int Lmax = set->Lmax;
    // refinement layers: the last R global layers, in FP32 on the CUDA cores, or
    // with FTSP2_REFINE_TC as BF16X3 tensor-core layers (nothing to refine when
    // the main layers are BF16X3 already)
    const bool refine_tc = (flags & FTSP2_REFINE_TC) && mode != FTSP2_FP32;
    const int R = (mode == FTSP2_FP32 || (refine_tc && mode == FTSP2_BF16X3)) ? 0 : refine_layers(flags);
    const int refine_from = Lmax - R;       // global layers >= this are refinement layers
    const bool all_simt = mode == FTSP2_FP32;
    const int fmt = fmt_of_mode(mode);
    const int rfmt = refine_tc ? OP_BF16X3 : OP_F32;
    int maxn = 0;
    for (int b = 0; b < nb; ++b) maxn = std::max(maxn, inst[b].n);

    int kinds[kMaxChains] = {CHAIN_FERMI, CHAIN_ENTROPY};
    if (want == 2) kinds[0] = CHAIN_ENTROPY;

    int* dstatus = reinterpret_cast<int*>(W + L.status);
    InstWork* iw = reinterpret_cast<InstWork*>(W + L.inst_work);
    Tile* tiles = reinterpret_cast<Tile*>(W + L.tiles);
    Tile* tiles_ref = L.ntiles_ref ? reinterpret_cast<Tile*>(W + L.tiles_ref) : nullptr;
    double* partials = reinterpret_cast<double*>(W + L.partials);

    SetupArgs sa;
    sa.H = dH;
    sa.inst = dInst;
    sa.nb = nb;
    sa.P = L.P;
    sa.Lmax = Lmax;
    sa.nchains = L.nchains;
    sa.BN = L.BN;
    sa.BM = L.BM;
    sa.BN_ref = 128;
    sa.BM_ref = 128;
    sa.models = models;
    sa.nmodels = (int)set->host.size();
    sa.flags = flags;
    sa.chain_kind[0] = kinds[0];
    sa.chain_kind[1] = kinds[1];
    sa.iw = iw;
    sa.tiles = tiles;
    sa.tiles_ref = tiles_ref;
    sa.rec = dRec;
    sa.status = dstatus;
    // FTSP2_LANCZOS: the FP32 copy of H lives in chain 0's Z plane, which the
    // initialisation overwrites only after the bounds are final
    sa.h32 = (flags & FTSP2_LANCZOS) ? reinterpret_cast<float*>(W + L.Z[0]) : nullptr;
    sa.done = reinterpret_cast<int*>(W + L.done);
    sa.done_layers = Lmax;
    launch_prep(sa, s);
    launch_gershgorin(sa, maxn, s);
    if (flags & FTSP2_LANCZOS) {
        LanczosArgs lz;
        lz.H32 = sa.h32;
        lz.inst = dInst;
        lz.iw = iw;
        lanczos_bind(lz, W + L.lanczos, nb, L.P);
        launch_lanczos(lz, maxn, di.sms, s);
    }
    launch_decide(sa, s);

    InitArgs ia;
    ia.H = dH;
    ia.inst = dInst;
    ia.rec = dRec;
    ia.models = models;
    ia.iw = iw;
    ia.nb = nb;
    ia.P = L.P;
    ia.nchains = L.nchains;
    ia.plane_elems = L.plane_elems;
    ia.main_fmt = fmt;
    ia.refine_fmt = rfmt;
    ia.refine_from = all_simt ? 0 : refine_from;
    ia.upper_only = (flags & FTSP2_FULL_OPERANDS) ? 0 : 1;
    for (int c = 0; c < kMaxChains; ++c) {
        ia.chain_kind[c] = kinds[c];
        ia.Z[c] = c < L.nchains ? reinterpret_cast<float*>(W + L.Z[c]) : nullptr;
        ia.A[c] = c < L.nchains ? reinterpret_cast<float*>(W + L.A[c]) : nullptr;
        for (int p = 0; p < 2; ++p) {
            ia.OP[c][p] = c < L.nchains ? W + L.OP[c][p] : nullptr;
            ia.OPR[c][p] = (c < L.nchains && L.OPR[c][p]) ? W + L.OPR[c][p] : nullptr;
        }
    }
    launch_init(ia, maxn, s);

    // tensor maps of both parities (tensor-core layers only)
    TmaMaps maps[2];
    if (!all_simt && refine_from > 0) {
        const CUtensorMapDataType dt = fmt == OP_F16X2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                       : fmt == OP_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        const int es = fmt == OP_TF32X3 ? 4 : 2;
        const int nsplit = fmt == OP_BF16X3 ? 3 : 2;
        const int bke = 128 / es;
        std::memset(maps, 0, sizeof(maps));
        for (int p = 0; p < 2; ++p)
            for (int c = 0; c < L.nchains; ++c)
                for (int sp = 0; sp < nsplit; ++sp) {
                    void* base = W + L.OP[c][p] + (size_t)sp * es * L.plane_elems;
                    if (!encode_map(&maps[p].a[c][sp], base, dt, es, L.P, nb, bke, kTileM)) return FTSP2_E_CUDA;
                    // transposed 64 x 64 panels of the upper triangle (16-bit planes)
                    if (es == 2 && !encode_map(&maps[p].t[c][sp], base, dt, es, L.P, nb, 64, 64))
                        return FTSP2_E_CUDA;
                }
    }
    // tensor maps of the BF16X3 refinement operands (FTSP2_REFINE_TC)
    TmaMaps mapsR[2];
    if (refine_tc && R > 0) {
        std::memset(mapsR, 0, sizeof(mapsR));
        for (int p = 0; p < 2; ++p)
            for (int c = 0; c < L.nchains; ++c)
                for (int sp = 0; sp < 3; ++sp) {
                    void* base = W + L.OPR[c][p] + (size_t)sp * 2 * L.plane_elems;
                    if (!encode_map(&mapsR[p].a[c][sp], base, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L.P, nb, 64, kTileM))
                        return FTSP2_E_CUDA;
                    if (!encode_map(&mapsR[p].t[c][sp], base, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, L.P, nb, 64, 64))
                        return FTSP2_E_CUDA;
                }
    }

    LayerArgs la;
    std::memset(&la, 0, sizeof(la));
    la.inst = dInst;
    la.rec = dRec;
    la.iw = iw;
    la.models = models;
    la.layers = layers;
    la.P = L.P;
    la.Lmax = Lmax;
    la.nchains = L.nchains;
    la.plane_elems = L.plane_elems;
    la.D = dD;
    la.partials = partials;
    la.status = dstatus;
    la.coef = set->d_coef;
    la.wait_ns = g_wait_ns.load();
    la.stall_layer = g_stall_layer.load();
    for (int c = 0; c < kMaxChains; ++c) {
        la.chain_kind[c] = kinds[c];
        la.Z[c] = c < L.nchains ? reinterpret_cast<float*>(W + L.Z[c]) : nullptr;
        la.A[c] = c < L.nchains ? reinterpret_cast<float*>(W + L.A[c]) : nullptr;
    }
    auto is_simt = [&](int g) { return all_simt || (g >= refine_from && !refine_tc); };
    auto is_rtc = [&](int g) { return refine_tc && g >= refine_from; };
    const int pair = all_simt ? 1 : tile_shape_choice(inst, nb, mode, want, flags, di.sms);
    // mean order n over the tensor-core tiles of the chosen shape (chunk policy)
    double mean_k = 0.0;
    {
        double wk = 0.0, wt = 0.0;
        const int T = pair ? 256 : 128;
        for (int b = 0; b < nb; ++b) {
            const double t = (double)host_tiles_of(inst[b].n, T, T);
            wt += t;
            wk += t * inst[b].n;
        }
        mean_k = wt > 0.0 ? wk / wt : 0.0;
    }
    int last_table = 0;
    // Operands of 16-bit tensor-core layers are stored as the upper triangle
    // plus the diagonal tile blocks when the layer that reads them can load the
    // rest transposed (FP16X2, BF16X3); the mirror is written everywhere before
    // an FP32 or TF32X3 layer.  init writes the same form for an instance whose
    // first layer is such a layer (ia.upper_only), so a layer's operands are
    // all of one form, whichever layer wrote them.
    const bool tc16_0 = !is_simt(0) && (is_rtc(0) || fmt == OP_F16X2 || fmt == OP_BF16X3);
    int prev_skips_mirror = (tc16_0 && ia.upper_only) ? 1 : 0;
    // a tensor-core layer that is not the last and whose successor has its
    // arithmetic: it writes operands of its own format (one kernel variant for
    // all such layers), so consecutive ones can share one multi-layer launch
    auto in_run = [&](int h) {
        return h < Lmax - 1 && !is_simt(h) && !is_simt(h + 1) && is_rtc(h) == is_rtc(h + 1);
    };
    for (int g = 0; g < Lmax; ++g) {
        const bool simt = is_simt(g);
        const bool next_simt = g + 1 < Lmax && is_simt(g + 1);
        const bool rtc = is_rtc(g);
        const bool next_rtc = g + 1 < Lmax && is_rtc(g + 1);
        const int lmode = rtc ? (int)FTSP2_BF16X3 : mode;   // arithmetic of this layer
        la.gl = g;
        la.nlayers = 1;
        la.last = g == Lmax - 1;
        // The last layers run with 64-element accumulation chunks: their rounding
        // reaches the output undamped (earlier errors are contracted by the
        // saturating later layers), and the entropy is linear in it for occupations
        // near 0 and 1.
        la.chunk_elems = chunk_elems_of(lmode, g, Lmax, mean_k);
        la.chunk_tail = la.chunk_elems;
        la.tail_from = INT_MAX;
        la.next_fmt = next_simt ? OP_F32 : (next_rtc ? OP_BF16X3 : fmt);
        const bool next_tc16 = !la.last && (la.next_fmt == OP_F16X2 || la.next_fmt == OP_BF16X3);
        la.mirror_all = (next_tc16 && !(flags & FTSP2_FULL_OPERANDS)) ? 0 : 1;
        la.lower_t = (!simt && prev_skips_mirror) ? 1 : 0;
        prev_skips_mirror = la.mirror_all ? 0 : 1;
        la.done_inst = reinterpret_cast<int*>(W + L.done);
        la.nb = nb;
        for (int c = 0; c < L.nchains; ++c) {
            const int rp = g & 1, wp = (g + 1) & 1;
            if (simt || rtc) la.opr[c] = all_simt ? W + L.OP[c][rp] : W + L.OPR[c][rp];
            else la.opr[c] = W + L.OP[c][rp];
            if (next_simt || next_rtc) la.opw[c] = all_simt ? W + L.OP[c][wp] : W + L.OPR[c][wp];
            else la.opw[c] = W + L.OP[c][wp];
            // write operands of layer g + 1 (same kind): parity (g + 2) & 1
            la.opw_alt[c] = (rtc ? W + L.OPR[c][rp] : W + L.OP[c][rp]);
        }
        if (dD == nullptr && la.last) la.D = nullptr;
        cudaError_t e;
        if (simt) {
            const bool use_ref = !all_simt;
            la.tiles = use_ref ? tiles_ref : tiles;
            la.ntiles = use_ref ? L.ntiles_ref : L.ntiles;
            const int grid = std::max(1, std::min(la.ntiles, di.sms * 4));
            e = launch_layer_simt(la, grid, s);
            last_table = use_ref ? 1 : 0;
        } else {
            la.tiles = pair ? tiles : tiles_ref;
            la.ntiles = pair ? L.ntiles : L.ntiles_ref;
            la.dtab = pair ? 0 : 1;
            const int units = std::max(1, std::min(la.ntiles, pair ? di.sms / 2 : di.sms));
            la.escr = pair && L.escr_ctas >= 2 * units ? reinterpret_cast<float*>(W + L.escr) : nullptr;
            // consecutive layers of this kind in one persistent launch when each
            // layer is only a few waves of tiles (at most 8), and every unit can
            // be resident at once (the launch's CTAs wait on one another).  With
            // more waves the idle tail of a launch is a small share, and runs
            // measured slower: at n = 8192 the busier GPU ran at a lower
            // power-capped clock (90.2 against 83.2 ms per solve), and on the
            // 512-instance ragged batch (71 waves) the units drifted apart
            // without a barrier per layer, the instances in flight at once
            // outgrew the L2, and the batch took 34.2 against 31.0 ms.
            int m = 1, lunits = units;
            if (!(flags & FTSP2_LAYER_LAUNCHES) && g_coop_ok.load() != 0 && !(capturing && g_coop_ok.load() != 1) &&
                la.ntiles <= 8 * units && in_run(g) &&
                (lmode == FTSP2_TF32X3 || la.lower_t == (la.mirror_all ? 0 : 1))) {
                while (g + m < Lmax && in_run(g + m)) ++m;
                if (m > 1) {
                    // at most the co-resident units (cluster placement may leave an SM out)
                    const bool defer = pair && la.escr != nullptr;
                    const int maxu = layer_tc_max_units(lmode, pair, defer);
                    if (maxu >= units) lunits = units;
                    else if (maxu >= (units * 9) / 10) lunits = maxu;
                    else m = 1;
                }
            }
            la.nlayers = m;
            if (m > 1) {
                // chunk schedule over the run: chunk_elems up to tail_from, chunk_tail after
                for (int h = g + 1; h < g + m; ++h) {
                    if (chunk_elems_of(lmode, h, Lmax, mean_k) != la.chunk_elems) {
                        la.tail_from = h;
                        la.chunk_tail = chunk_elems_of(lmode, h, Lmax, mean_k);
                        break;
                    }
                }
            }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            {
                std::lock_guard<std::mutex> lk(g_prof_mu);
                if (g_prof_on && !capturing && cudaEventCreate(&e0) == cudaSuccess &&
                    cudaEventCreate(&e1) == cudaSuccess) {
                    cudaEventRecord(e0, s);
                } else {
                    e0 = e1 = nullptr;
                }
            }
            const TmaMaps& m0 = rtc ? mapsR[g & 1] : maps[g & 1];
            const TmaMaps& m1 = rtc ? mapsR[(g + 1) & 1] : maps[(g + 1) & 1];
            e = launch_layer_tc(lmode, la, m0, m1, m > 1 ? lunits : units, pair, s);
            if (m > 1) {
                if (e != cudaSuccess && !capturing) {
                    // multi-layer launches refused here: one launch per layer from now on
                    cudaGetLastError();
                    g_coop_ok.store(0);
                    la.nlayers = m = 1;
                    la.tail_from = INT_MAX;
                    e = launch_layer_tc(lmode, la, m0, m1, units, pair, s);
                } else if (e == cudaSuccess) {
                    g_coop_ok.store(1);
                }
            }
            if (e0) {
                cudaEventRecord(e1, s);
                std::lock_guard<std::mutex> lk(g_prof_mu);
                g_prof_events.push_back(ProfEvent{e0, e1, m});
            }
            last_table = pair ? 0 : 1;
            g += m - 1;     // the run's remaining layers are done
        }
        if (e != cudaSuccess) return FTSP2_E_CUDA;
    }
    FinalArgs fa;
    fa.inst = dInst;
    fa.rec = dRec;
    fa.models = models;
    fa.iw = iw;
    fa.partials = partials;
    fa.table = last_table;
    fa.nb = nb;
    fa.nchains = L.nchains;
    fa.chain_kind[0] = kinds[0];
    fa.chain_kind[1] = kinds[1];
    fa.trace = (want & 1) ? dTrace : nullptr;
    fa.S = (want & 2) ? dS : nullptr;
    fa.status = dstatus;
    launch_finalize(fa, s);
    if (cudaGetLastError() != cudaSuccess) return FTSP2_E_CUDA;
    if (flags & FTSP2_SYNC) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return FTSP2_E_CUDA;
        std::vector<ftsp2_rescale_rec> h(nb);
        if (cudaMemcpy(h.data(), dRec, sizeof(ftsp2_rescale_rec) * nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            return FTSP2_E_CUDA;
        int worst = FTSP2_OK;
        for (auto& r : h)
            if (r.status != FTSP2_OK) worst = r.status;
        return (ftsp2_status)worst;
    }
    return FTSP2_OK;
}

// ------------------------------------------------------------------------------
// training driver
// ------------------------------------------------------------------------------
struct TrainLayout {
    size_t M, R, Rh, G, part, apart, v, out, amax;
    size_t X;             // the sample points (built by the library)
    size_t total;
    int nchunks;
};

static TrainLayout train_layout(int ns, int L) {
    TrainLayout t;
    const int np = 4 * L, m = np + 1;
    t.nchunks = 64;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    t.M = take(sizeof(double) * (size_t)m * ns);
    t.R = take(sizeof(double) * ns);
    t.Rh = take(sizeof(double) * ns);
    t.G = take(sizeof(double) * (size_t)m * m);
    t.part = take(sizeof(double) * (size_t)t.nchunks * m * m);
    t.apart = take(sizeof(double) * (size_t)((ns + 255) / 256) * np);
    t.v = take(sizeof(double) * np);
    t.out = take(sizeof(double) * np);
    t.amax = take(sizeof(double) * 80);
    t.X = take(sizeof(double) * ns);
    t.total = off;
    return t;
}

// Cholesky solve of (A) x = b for a symmetric positive definite A (n x n, FP64).
static bool chol_solve(std::vector<double> A, int n, const std::vector<double>& b, std::vector<double>& x) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        d = std::sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / d;
        }
    }
    x = b;
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= A[(size_t)i * n + k] * x[k];
        x[i] = s / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= A[(size_t)k * n + i] * x[k];
        x[i] = s / A[(size_t)i * n + i];
    }
    return true;
}

}  // namespace ftsp2

using namespace ftsp2;

extern "C" {

const char* ftsp2_status_string(ftsp2_status s) {
    switch (s) {
        case FTSP2_OK: return "ok";
        case FTSP2_E_ARG: return "invalid argument";
        case FTSP2_E_CUDA: return "CUDA error";
        case FTSP2_E_WORKSPACE: return "workspace too small or misaligned";
        case FTSP2_E_VALIDITY: return "beta' outside every model's region of validity";
        case FTSP2_E_NONFINITE: return "non-finite input or result";
        case FTSP2_E_TIMEOUT: return "device-side wait timed out";
        case FTSP2_E_NOMODEL: return "no model";
        case FTSP2_E_UNSUPPORTED: return "unsupported device or mode";
    }
    return "unknown status";
}

uint64_t ftsp2_kernel_launch_count(void) { return g_launches.load(); }

ftsp2_status ftsp2_set_wait_limit_ns(uint64_t ns) {
    if (ns < 100000ull || ns > 60000000000ull) return FTSP2_E_ARG;
    g_wait_ns.store(ns);
    return FTSP2_OK;
}

uint64_t ftsp2_wait_limit_ns(void) { return g_wait_ns.load(); }

ftsp2_status ftsp2_debug_stall_layer(int layer) {
    if (layer < -1 || layer >= kMaxLayers) return FTSP2_E_ARG;
    g_stall_layer.store(layer);
    return FTSP2_OK;
}

ftsp2_status ftsp2_profile_layers(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
    return FTSP2_OK;
}

ftsp2_status ftsp2_profile_read(double* total_ms, uint64_t* launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double sum = 0.0;
    uint64_t n = 0;
    ftsp2_status st = FTSP2_OK;
    for (auto& pr : g_prof_events) {
        float ms = 0.f;
        if (cudaEventSynchronize(pr.e1) != cudaSuccess || cudaEventElapsedTime(&ms, pr.e0, pr.e1) != cudaSuccess)
            st = FTSP2_E_CUDA;
        else {
            sum += ms;
            n += (uint64_t)pr.layers;
        }
        cudaEventDestroy(pr.e0);
        cudaEventDestroy(pr.e1);
    }
    g_prof_events.clear();
    if (total_ms) *total_ms = sum;
    if (launches) *launches = n;
    return st;
}

ftsp2_status ftsp2_model_set_create(const ftsp2_table* tabs, int ntab, ftsp2_model_set** out) {
    if (!out) return FTSP2_E_ARG;
    *out = nullptr;
    if (!tabs || ntab < 1) return FTSP2_E_NOMODEL;
    auto* s = new ftsp2_model_set();
    for (int i = 0; i < ntab; ++i) {
        const ftsp2_table& t = tabs[i];
        const int LS = t.theta_entropy ? t.L_entropy : t.L;
        // a Skip-SP2 table carries an output row: at most kMaxLayers rows in
        // all; a Max-SP2 table keeps every layer: at most kMaxMaxLayers
        const int lmax = t.family == FTSP2_FAMILY_SKIP ? kMaxLayers - 1
                         : t.family == FTSP2_FAMILY_MAX ? kMaxMaxLayers : kMaxLayers;
        if (t.L < 1 || t.L > lmax || LS < 1 || LS > lmax || !t.theta || !(t.beta0 > 0) ||
            !(t.mu0 > 0 && t.mu0 < 1) || !std::isfinite(t.alpha)) {
            delete s;
            return FTSP2_E_ARG;
        }
        if (t.family != FTSP2_FAMILY_MLSP2 && t.family != FTSP2_FAMILY_SKIP && t.family != FTSP2_FAMILY_MAX) {
            delete s;
            return FTSP2_E_ARG;
        }
        HostModel h;
        h.L = t.L;
        h.LS = LS;
        h.family = t.family;
        h.beta0 = t.beta0;
        h.mu0 = t.mu0;
        h.alpha = t.alpha;
        if (t.family == FTSP2_FAMILY_MAX) {
            h.th.assign(t.theta, t.theta + max_nparams(t.L));
            if (t.theta_entropy) h.thS.assign(t.theta_entropy, t.theta_entropy + max_nparams(LS));
            s->has_max = true;
            s->planes = std::max(s->planes, std::max(t.L, LS) + 1);
        } else {
            const int rows = t.family == FTSP2_FAMILY_SKIP ? 1 : 0;   // the output row of Skip-SP2
            h.th.assign(t.theta, t.theta + 4 * (t.L + rows));
            if (t.theta_entropy) h.thS.assign(t.theta_entropy, t.theta_entropy + 4 * (LS + rows));
        }
        for (double v : h.th)
            if (!std::isfinite(v)) { delete s; return FTSP2_E_ARG; }
        for (double v : h.thS)
            if (!std::isfinite(v)) { delete s; return FTSP2_E_ARG; }
        s->Lmax = std::max(s->Lmax, std::max(h.L, h.LS));
        s->host.push_back(std::move(h));
    }
    const ftsp2_status st = upload_models(s);
    if (st != FTSP2_OK) {
        ftsp2_model_set_destroy(s);
        return st;
    }
    *out = s;
    return FTSP2_OK;
}

ftsp2_status ftsp2_model_set_builtin(ftsp2_model_set** out) {
    ftsp2_table t;
    std::memset(&t, 0, sizeof(t));
    t.family = FTSP2_FAMILY_MLSP2;
    t.L = 26;
    t.L_entropy = 0;
    t.beta0 = 1500.0;
    t.mu0 = 1.0 / 3.0;
    t.alpha = 0.842704;
    t.theta = &kPrinted[0][0];
    t.theta_entropy = nullptr;
    return ftsp2_model_set_create(&t, 1, out);
}

void ftsp2_model_set_destroy(ftsp2_model_set* s) {
    if (!s) return;
    if (s->d_mem) cudaFree(s->d_mem);
    delete s;
}

ftsp2_status ftsp2_model_set_info(const ftsp2_model_set* s, int* ntab, int* max_layers) {
    if (!s) return FTSP2_E_ARG;
    if (ntab) *ntab = (int)s->host.size();
    if (max_layers) *max_layers = s->Lmax;
    return FTSP2_OK;
}

ftsp2_status ftsp2_model_set_table(const ftsp2_model_set* s, int idx, int* L, double* theta_out, double* beta0,
                                   double* mu0, double* alpha) {
    if (!s || idx < 0 || idx >= (int)s->host.size()) return FTSP2_E_ARG;
    const HostModel& h = s->host[idx];
    if (L) *L = h.L;
    if (theta_out) std::copy(h.th.begin(), h.th.end(), theta_out);
    if (beta0) *beta0 = h.beta0;
    if (mu0) *mu0 = h.mu0;
    if (alpha) *alpha = h.alpha;
    return FTSP2_OK;
}

ftsp2_status ftsp2_workspace_size_set(const ftsp2_instance* inst, int nb, const ftsp2_model_set* set,
                                      ftsp2_mode mode, int want, size_t* bytes) {
    if (!bytes) return FTSP2_E_ARG;
    if (!set || set->host.empty()) return FTSP2_E_NOMODEL;
    Layout L;
    const ftsp2_status st = plan(inst, nb, mode, want, FTSP2_REFINE2 | FTSP2_REFINE_TC | FTSP2_EPI_DEFERRED, L,
                                 set->planes);
    if (st != FTSP2_OK) return st;
    *bytes = L.total;
    return FTSP2_OK;
}

ftsp2_status ftsp2_workspace_size(const ftsp2_instance* inst, int nb, ftsp2_mode mode, int want, size_t* bytes) {
    if (!bytes) return FTSP2_E_ARG;
    Layout L;
    // sized for the largest refinement setting so one workspace serves every flag
    const ftsp2_status st = plan(inst, nb, mode, want, FTSP2_REFINE2 | FTSP2_REFINE_TC | FTSP2_EPI_DEFERRED, L);
    if (st != FTSP2_OK) return st;
    *bytes = L.total;
    return FTSP2_OK;
}

static size_t rescale_ws_bytes(int nb) { return 1024 + align_up(sizeof(InstWork) * (size_t)nb, 1024); }

ftsp2_status ftsp2_rescale_workspace_size(int nb, size_t* bytes) {
    if (!bytes || nb < 1) return FTSP2_E_ARG;
    *bytes = rescale_ws_bytes(nb);
    return FTSP2_OK;
}

ftsp2_status ftsp2_rescale(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, int flags, ftsp2_rescale_rec* dRec, void* ws,
                           size_t ws_bytes, void* stream) {
    if (!set || set->host.empty()) return FTSP2_E_NOMODEL;
    if (!dH || !inst || !dInst || !dRec || nb < 1 || !ws) return FTSP2_E_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % 1024 != 0 || ws_bytes < rescale_ws_bytes(nb)) return FTSP2_E_WORKSPACE;
    DeviceInfo di;
    ftsp2_status st = device_info(di);
    if (st != FTSP2_OK) return st;
    int maxn = 0;
    for (int b = 0; b < nb; ++b) {
        if (inst[b].n < 1 || inst[b].offset < 0) return FTSP2_E_ARG;
        maxn = std::max(maxn, inst[b].n);
    }
    const int P = (int)align_up((size_t)maxn, kPad);
    // FTSP2_LANCZOS: Lanczos buffers, then the FP32 copy of H (P x P slab per instance)
    const size_t h32_elems = (size_t)nb * P * P;
    const size_t lz_off = rescale_ws_bytes(nb), h32_off = lz_off + lanczos_ws_bytes(nb, P);
    if ((flags & FTSP2_LANCZOS) && ws_bytes < h32_off + sizeof(float) * h32_elems) return FTSP2_E_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* W = static_cast<uint8_t*>(ws);
    SetupArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.H = dH;
    sa.inst = dInst;
    sa.nb = nb;
    sa.P = P;
    sa.Lmax = set->Lmax;
    sa.nchains = 1;
    sa.BN = 128;
    sa.BM = 128;
    sa.models = set->d_models[0];
    sa.nmodels = (int)set->host.size();
    sa.flags = flags;
    sa.chain_kind[0] = CHAIN_FERMI;
    sa.iw = reinterpret_cast<InstWork*>(W + 1024);
    sa.tiles = nullptr;
    sa.tiles_ref = nullptr;
    sa.rec = dRec;
    sa.status = reinterpret_cast<int*>(W);
    sa.h32 = (flags & FTSP2_LANCZOS) ? reinterpret_cast<float*>(W + h32_off) : nullptr;
    launch_prep(sa, s);
    launch_gershgorin(sa, maxn, s);
    if (flags & FTSP2_LANCZOS) {
        LanczosArgs lz;
        lz.H32 = sa.h32;
        lz.inst = dInst;
        lz.iw = sa.iw;
        lanczos_bind(lz, W + lz_off, nb, P);
        launch_lanczos(lz, maxn, di.sms, s);
    }
    launch_decide(sa, s);
    if (cudaGetLastError() != cudaSuccess) return FTSP2_E_CUDA;
    if (flags & FTSP2_SYNC) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return FTSP2_E_CUDA;
        std::vector<ftsp2_rescale_rec> h(nb);
        if (cudaMemcpy(h.data(), dRec, sizeof(ftsp2_rescale_rec) * nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            return FTSP2_E_CUDA;
        int worst = FTSP2_OK;
        for (auto& r : h)
            if (r.status != FTSP2_OK) worst = r.status;
        return (ftsp2_status)worst;
    }
    return FTSP2_OK;
}

ftsp2_status ftsp2_density(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, ftsp2_mode mode, int flags, float* dD, double* dTrace,
                           ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes, void* stream) {
    return run(dH, inst, dInst, nb, set, mode, flags, 1, dD, dTrace, nullptr, dRec, ws, ws_bytes, stream);
}

ftsp2_status ftsp2_entropy(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst, int nb,
                           const ftsp2_model_set* set, ftsp2_mode mode, int flags, double* dS,
                           ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes, void* stream) {
    return run(dH, inst, dInst, nb, set, mode, flags, 2, nullptr, nullptr, dS, dRec, ws, ws_bytes, stream);
}

ftsp2_status ftsp2_density_entropy(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst,
                                   int nb, const ftsp2_model_set* set, ftsp2_mode mode, int flags, float* dD,
                                   double* dTrace, double* dS, ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes,
                                   void* stream) {
    if (!dS) return ftsp2_density(dH, inst, dInst, nb, set, mode, flags, dD, dTrace, dRec, ws, ws_bytes, stream);
    if (!dD && !dTrace)
        return ftsp2_entropy(dH, inst, dInst, nb, set, mode, flags, dS, dRec, ws, ws_bytes, stream);
    return run(dH, inst, dInst, nb, set, mode, flags, 3, dD, dTrace, dS, dRec, ws, ws_bytes, stream);
}

ftsp2_status ftsp2_density_mu(const double* dH, const ftsp2_instance* inst, ftsp2_instance* dInst, int nb,
                              const double* dNocc, const ftsp2_model_set* set, ftsp2_mode mode, int flags,
                              int iterations, double tol, float* dD, double* dTrace, double* dS,
                              ftsp2_rescale_rec* dRec, int32_t* dSteps, void* ws, size_t ws_bytes, void* stream) {
    if (iterations < 0 || iterations > 64 || !(tol >= 0.0) || nb < 1 || !inst) return FTSP2_E_ARG;
    if (!dNocc || !dTrace || !dSteps || !dInst) return FTSP2_E_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(dSteps, 0, sizeof(int32_t) * (size_t)nb, s) != cudaSuccess) return FTSP2_E_CUDA;
    const int quiet = flags & ~FTSP2_SYNC;
    for (int it = 0;; ++it) {
        const bool last = it == iterations;
        // evaluations before the last need only the density and its traces
        const ftsp2_status st = last && dS
                                    ? run(dH, inst, dInst, nb, set, mode, flags, 3, dD, dTrace, dS, dRec, ws, ws_bytes,
                                          stream)
                                    : run(dH, inst, dInst, nb, set, mode, last ? flags : quiet, 1, dD, dTrace,
                                          nullptr, dRec, ws, ws_bytes, stream);
        if (last || st != FTSP2_OK) return st;
        MuArgs ma;
        ma.inst = dInst;
        ma.rec = dRec;
        ma.trace = dTrace;
        ma.nocc = dNocc;
        ma.steps = dSteps;
        ma.tol = tol;
        ma.nb = nb;
        launch_mu_update(ma, s);
        if (cudaGetLastError() != cudaSuccess) return FTSP2_E_CUDA;
    }
}

static int want_of(const float* dD, const double* dTrace, const double* dS) {
    if (!dS) return 1;
    if (!dD && !dTrace) return 2;
    return 3;
}

ftsp2_status ftsp2_autotune(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst, int nb,
                            const ftsp2_model_set* set, ftsp2_mode mode, int flags, float* dD, double* dTrace,
                            double* dS, ftsp2_rescale_rec* dRec, void* ws, size_t ws_bytes, int reps, int* choice,
                            float* ms, void* stream) {
    if (reps < 1 || !choice) return FTSP2_E_ARG;
    if (nb < 1 || !inst) return FTSP2_E_ARG;
    if (ms) ms[0] = ms[1] = 0.f;
    const int base = flags & ~(FTSP2_PAIR_TILES | FTSP2_SINGLE_TILES | FTSP2_SYNC);
    if (mode == FTSP2_FP32) {
        *choice = -1;
        return ftsp2_density_entropy(dH, inst, dInst, nb, set, mode, base | FTSP2_SYNC, dD, dTrace, dS, dRec, ws,
                                     ws_bytes, stream);
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FTSP2_E_CUDA;
    }
    float t[2] = {0.f, 0.f};
    ftsp2_status st = FTSP2_OK;
    for (int shape = 0; shape < 2 && st == FTSP2_OK; ++shape) {
        const int f = base | (shape ? FTSP2_PAIR_TILES : FTSP2_SINGLE_TILES);
        // untimed run with FTSP2_SYNC: surfaces per-instance errors once
        st = ftsp2_density_entropy(dH, inst, dInst, nb, set, mode, f | FTSP2_SYNC, dD, dTrace, dS, dRec, ws,
                                   ws_bytes, stream);
        if (st != FTSP2_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = FTSP2_E_CUDA; break; }
        for (int r = 0; r < reps && st == FTSP2_OK; ++r)
            st = ftsp2_density_entropy(dH, inst, dInst, nb, set, mode, f, dD, dTrace, dS, dRec, ws, ws_bytes,
                                       stream);
        if (st != FTSP2_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t[shape], e0, e1) != cudaSuccess) {
            st = FTSP2_E_CUDA;
            break;
        }
        t[shape] /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FTSP2_OK) return st;
    const int pick = t[1] <= t[0] ? 1 : 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[batch_signature(inst, nb, mode, want_of(dD, dTrace, dS), base)] = pick;
    }
    *choice = pick;
    if (ms) {
        ms[0] = t[0];
        ms[1] = t[1];
    }
    return FTSP2_OK;
}

ftsp2_status ftsp2_tile_shape(const ftsp2_instance* inst, int nb, ftsp2_mode mode, int want, int flags, int* shape,
                              int* from_tuner) {
    if (!inst || nb < 1 || !shape || want < 1 || want > 3) return FTSP2_E_ARG;
    if (from_tuner) *from_tuner = 0;
    if (mode == FTSP2_FP32) {
        *shape = -1;
        return FTSP2_OK;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FTSP2_E_CUDA;
    *shape = tile_shape_choice(inst, nb, mode, want, flags, sms, from_tuner);
    return FTSP2_OK;
}

ftsp2_status ftsp2_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return FTSP2_OK;
}

}  // extern "C"

namespace ftsp2 {

// ---- density without any allocation ------------------------------------------
//
// Some callers cannot allocate device memory at the point where they need a
// density matrix: code that runs while a stream is being captured into a CUDA
// graph (an allocation there breaks or invalidates the capture), plug-ins that
// live inside a host application owning every device allocation, and
// real-time loops that forbid the cost and possible synchronisation of
// cudaMalloc.  ftsp2_density_noalloc serves them: it runs the same kernels as
// ftsp2_density but takes its scratch (the workspace of ftsp2_density) from
// the fixed device array below instead of from the caller.

// 8 MiB of scratch in the library image.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kNoallocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and
// cached; the lookup allocates nothing.  The lookup may load the module, which
// must not happen inside a stream capture: a first call on a device made while
// `stream` is capturing is refused (FTSP2_E_ARG) before the lookup.
static ftsp2_status noalloc_scratch(void** ws, size_t* bytes, cudaStream_t stream) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static void* addr[kMaxDevices] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FTSP2_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FTSP2_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return FTSP2_E_CUDA;
        if (cap != cudaStreamCaptureStatusNone) return FTSP2_E_ARG;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FTSP2_E_CUDA;
        addr[dev] = p;
    }
    // the hot path wants a 1024-byte aligned workspace
    const uintptr_t base = reinterpret_cast<uintptr_t>(addr[dev]);
    const uintptr_t aligned = (base + 1023) & ~uintptr_t(1023);
    *ws = reinterpret_cast<void*>(aligned);
    *bytes = kNoallocScratchBytes - (size_t)(aligned - base);
    return FTSP2_OK;
}

}  // namespace ftsp2

extern "C" {

ftsp2_status ftsp2_density_noalloc(const double* dH, const ftsp2_instance* inst, const ftsp2_instance* dInst,
                                   int nb, const ftsp2_model_set* set, ftsp2_mode mode, int flags, float* dD,
                                   double* dTrace, ftsp2_rescale_rec* dRec, void* stream) {
    // FTSP2_SYNC would need a host buffer for the records: not offered here.
    if (flags & FTSP2_SYNC) return FTSP2_E_ARG;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    const ftsp2_status st = noalloc_scratch(&ws, &ws_bytes, static_cast<cudaStream_t>(stream));
    if (st != FTSP2_OK) return st;
    // run() checks the plan against ws_bytes and returns FTSP2_E_WORKSPACE,
    // before launching anything, when the batch needs more scratch than the array.
    return run(dH, inst, dInst, nb, set, mode, flags, 1, dD, dTrace, nullptr, dRec, ws, ws_bytes, stream);
}

size_t ftsp2_train_workspace_size(int nsamples, int L) {
    if (nsamples < 1 || L < 1 || L > kMaxLayers) return 0;
    return train_layout(nsamples, L).total;
}

static ftsp2_status load_theta(int L, const double* theta, ThetaParam& tp) {
    if (!theta || L < 1 || L > kMaxLayers) return FTSP2_E_ARG;
    std::memset(&tp, 0, sizeof(tp));
    for (int i = 0; i < 4 * L; ++i) {
        if (!std::isfinite(theta[i])) return FTSP2_E_ARG;
        tp.v[i] = theta[i];
    }
    return FTSP2_OK;
}

ftsp2_status ftsp2_train_residual_jacobian(int target, double beta0, double mu0, int L, double alpha,
                                           const double* theta, const double* dX, int nsamples, double* dR,
                                           double* dJ, void* stream) {
    // dJ: the augmented parameter-major Jacobian M
    if ((target != FTSP2_TARGET_FERMI && target != FTSP2_TARGET_ENTROPY) || !dX || !dR || nsamples < 1)
        return FTSP2_E_ARG;
    ThetaParam tp;
    ftsp2_status st = load_theta(L, theta, tp);
    if (st != FTSP2_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = dJ ? launch_train_fwd_jac(target, beta0, mu0, L, alpha, tp, dX, nsamples, dR, dJ, s)
                       : launch_train_residual(target, beta0, mu0, L, alpha, tp, dX, nsamples, dR, s);
    return from_cuda(e);
}

ftsp2_status ftsp2_train_normal_equations(const double* dM, int nsamples, int L, double* dG, void* dWork,
                                          size_t work_bytes, void* stream) {
    if (!dM || !dG || !dWork || nsamples < 1 || L < 1 || L > kMaxLayers) return FTSP2_E_ARG;
    const TrainLayout tl = train_layout(nsamples, L);
    if (work_bytes < tl.total) return FTSP2_E_WORKSPACE;
    double* dPart = reinterpret_cast<double*>(static_cast<uint8_t*>(dWork) + tl.part);
    return from_cuda(launch_train_gram(dM, nsamples, 4 * L, dG, dPart, tl.nchunks, static_cast<cudaStream_t>(stream)));
}

// ---- parameterisations of the trained table ---------------------------------
// The LM loop runs on a parameter vector p.  Eq. mlsp2 tables: p = theta (4L).
// One-term form (Eq. mlsp2_alt): p = (t_01, t_02, ..., t_L1, t_L2) (2L + 2),
// theta(p) by ftsp2_alt_to_mlsp2 and the Jacobian P = d theta / d p, so that
// J_p = J P and the reductions transform as P^T (J^T J) P and P^T (J^T r).
// Skip-SP2 tables (FORM_SKIP): p = the table itself, 4L + 2 entries (layer
// rows, then A_0 and gamma_L), with its own forward/Jacobian kernel.
// Max-SP2 tables (FORM_MAX): p = the flat table, L (L + 5) / 2 + 2 entries.
// Skip-SP2 with k stored layers and K accumulators (FORM_SKIPK): p = (alpha
// (L x (k + 1), the constant last), beta (L x K), gamma (L x K), A_{0,1},
// gamma_L), (1 + k + 2K) L + 2 entries, the other initial accumulators zero;
// theta(p) = its Max-SP2 embedding (ftsp2_skip_to_max) and P its exact
// Jacobian (the embedding is affine in each single parameter).
enum { FORM_MLSP2 = 0, FORM_ALT = 1, FORM_SKIP = 2, FORM_MAX = 3, FORM_SKIPK = 4 };

struct FormDims {
    int k = 1, K = 1;          // FORM_SKIPK only
};

static int form_params(int form, int L, const FormDims& fd = FormDims()) {
    switch (form) {
        case FORM_ALT: return 2 * L + 2;
        case FORM_SKIP: return 4 * L + 2;
        case FORM_MAX: return max_nparams(L);
        case FORM_SKIPK: return (1 + fd.k + 2 * fd.K) * L + 2;
        default: return 4 * L;
    }
}
static int form_theta_dim(int form, int L) {
    return form == FORM_SKIP ? 4 * L + 2 : (form == FORM_MAX || form == FORM_SKIPK) ? max_nparams(L) : 4 * L;
}
static int form_family(int form) {
    return form == FORM_SKIP ? FTSP2_FAMILY_SKIP
                             : (form == FORM_MAX || form == FORM_SKIPK) ? FTSP2_FAMILY_MAX : FTSP2_FAMILY_MLSP2;
}

// Max-SP2 embedding of a FORM_SKIPK parameter vector
static ftsp2_status skipk_theta(int L, const FormDims& fd, const double* p, double* th) {
    const int k = fd.k, K = fd.K;
    const double* al = p;
    const double* be = al + L * (k + 1);
    const double* ga = be + L * K;
    std::vector<double> A0(std::max(K, 1), 0.0);
    A0[0] = ga[L * K];
    return ftsp2_skip_to_max(L, k, K, al, K ? be : nullptr, K ? ga : nullptr, K ? A0.data() : nullptr,
                             ga[L * K + 1], th);
}

// d theta / d p of FORM_SKIPK (nt x np, row-major), written out from the
// embedding: delta_i = alpha_{i,k} + beta_{i,1} A_{0,1},
// theta_{i,j} = sum_l beta_{i,l} gamma_{j,l} [j < i] + alpha_{i,i-j} [i - j < k],
// gamma_j = sum_l gamma_{j,l}, c = A_{0,1}, gamma_L.
static void skipk_jacobian(int L, const FormDims& fd, const double* p, std::vector<double>& P) {
    const int k = fd.k, K = fd.K, np = form_params(FORM_SKIPK, L, fd), nt = max_nparams(L);
    const int pa = 0, pb = L * (k + 1), pg = pb + L * K, pA = pg + L * K, pL = pA + 1;
    P.assign((size_t)nt * np, 0.0);
    auto at = [&](int row, int col) -> double& { return P[(size_t)row * np + col]; };
    int o = 0;
    for (int i = 0; i < L; ++i) {
        at(o, pa + i * (k + 1) + k) = 1.0;
        if (K > 0) {
            at(o, pb + i * K) += p[pA];
            at(o, pA) += p[pb + i * K];
        }
        for (int l = 0; l < K; ++l) at(o + 1, pg + i * K + l) = 1.0;
        for (int j = 0; j <= i; ++j) {
            const int row = o + 2 + j;
            if (j < i)
                for (int l = 0; l < K; ++l) {
                    at(row, pb + i * K + l) += p[pg + j * K + l];
                    at(row, pg + j * K + l) += p[pb + i * K + l];
                }
            if (i - j < k) at(row, pa + i * (k + 1) + (i - j)) += 1.0;
        }
        o += i + 3;
    }
    at(o, pA) = 1.0;
    at(o + 1, pL) = 1.0;
}

static void alt_rows(int L, const double* alt, double* th) {
    for (int i = 0; i < L; ++i) {
        const double t1 = alt[2 * i], t2 = alt[2 * i + 1];
        th[4 * i + 0] = 1.0;
        th[4 * i + 1] = 2.0 * t1;
        th[4 * i + 2] = t1 * t1;
        th[4 * i + 3] = t2;
    }
    const double u = alt[2 * L], w = alt[2 * L + 1];
    double* last = th + 4 * (L - 1);
    last[0] *= w;
    last[1] *= w;
    last[2] = last[2] * w + u;
}

// P (nt x np, row-major) at p
static void form_jacobian(int form, int L, const double* p, std::vector<double>& P, const FormDims& fd) {
    if (form == FORM_SKIPK) {
        skipk_jacobian(L, fd, p, P);
        return;
    }
    const int np = form_params(form, L, fd), nt = form_theta_dim(form, L);
    P.assign((size_t)nt * np, 0.0);
    if (form != FORM_ALT) {
        for (int i = 0; i < nt; ++i) P[(size_t)i * np + i] = 1.0;
        return;
    }
    const double w = p[2 * L + 1];
    for (int i = 0; i < L; ++i) {
        const double t1 = p[2 * i];
        const double sc = i == L - 1 ? w : 1.0;
        P[(size_t)(4 * i + 1) * np + 2 * i] = 2.0 * sc;
        P[(size_t)(4 * i + 2) * np + 2 * i] = 2.0 * t1 * sc;
        P[(size_t)(4 * i + 3) * np + 2 * i + 1] = 1.0;
    }
    const double t1 = p[2 * (L - 1)];
    const int r = 4 * (L - 1);
    P[(size_t)(r + 0) * np + 2 * L + 1] = 1.0;
    P[(size_t)(r + 1) * np + 2 * L + 1] = 2.0 * t1;
    P[(size_t)(r + 2) * np + 2 * L + 1] = t1 * t1;
    P[(size_t)(r + 2) * np + 2 * L] = 1.0;
}

static ftsp2_status form_theta(int form, int L, const double* p, ThetaParam& tp, const FormDims& fd) {
    if (form == FORM_MLSP2) return load_theta(L, p, tp);
    if (form == FORM_MAX || form == FORM_SKIPK) {
        if (!p || L < 1 || L > kMaxMaxLayers) return FTSP2_E_ARG;
        std::memset(&tp, 0, sizeof(tp));
        const int np = form_params(form, L, fd);
        for (int i = 0; i < np; ++i)
            if (!std::isfinite(p[i])) return FTSP2_E_ARG;
        if (form == FORM_MAX) {
            std::copy(p, p + np, tp.v);
            return FTSP2_OK;
        }
        return skipk_theta(L, fd, p, tp.v);
    }
    if (form == FORM_SKIP) {
        if (!p || L < 1 || L > kMaxLayers - 1) return FTSP2_E_ARG;
        std::memset(&tp, 0, sizeof(tp));
        for (int i = 0; i < 4 * L + 2; ++i) {
            if (!std::isfinite(p[i])) return FTSP2_E_ARG;
            tp.v[i] = p[i];
        }
        return FTSP2_OK;
    }
    if (!p || L < 1 || L > kMaxLayers) return FTSP2_E_ARG;
    for (int i = 0; i < 2 * L + 2; ++i)
        if (!std::isfinite(p[i])) return FTSP2_E_ARG;
    std::memset(&tp, 0, sizeof(tp));
    alt_rows(L, p, tp.v);
    return FTSP2_OK;
}

// Levenberg-Marquardt (optionally geodesic-accelerated) on p; residuals, the
// Jacobian of theta and J^T J, J^T r run on the GPU, the rest on the host.
// Rows argument of train_layout for a form: room for its nt + 1 columns
static int form_layout_rows(int form, int L) {
    if (form == FORM_SKIP) return L + 1;
    if (form == FORM_MAX || form == FORM_SKIPK) return (max_nparams(L) + 3) / 4;
    return L;
}

static ftsp2_status lm_train(int form, int target, double beta0, double mu0, int L, double alpha, const double* dX,
                             int nsamples, int iterations, int accel, const double* p_init, double* p_out,
                             ftsp2_train_report* rep, void* dWork, size_t work_bytes, void* stream,
                             const FormDims& fd = FormDims()) {
    if ((target != FTSP2_TARGET_FERMI && target != FTSP2_TARGET_ENTROPY) || !dX || nsamples < 1 || !p_out ||
        !dWork || iterations < 0 || !p_init)
        return FTSP2_E_ARG;
    const int np = form_params(form, L, fd), nt = form_theta_dim(form, L);
    const int fam = form_family(form);
    std::vector<double> p(p_init, p_init + np);
    ThetaParam tp;
    ftsp2_status st = form_theta(form, L, p.data(), tp, fd);
    if (st != FTSP2_OK) return st;
    const TrainLayout tl = train_layout(nsamples, form_layout_rows(form, L));
    if (work_bytes < tl.total) return FTSP2_E_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* W = static_cast<uint8_t*>(dWork);
    double* dM = reinterpret_cast<double*>(W + tl.M);
    double* dRr = reinterpret_cast<double*>(W + tl.R);
    double* dRh = reinterpret_cast<double*>(W + tl.Rh);
    double* dG = reinterpret_cast<double*>(W + tl.G);
    double* dPart = reinterpret_cast<double*>(W + tl.part);
    double* dAp = reinterpret_cast<double*>(W + tl.apart);
    double* dV = reinterpret_cast<double*>(W + tl.v);
    double* dOut = reinterpret_cast<double*>(W + tl.out);
    double* dAm = reinterpret_cast<double*>(W + tl.amax);
    const int mt = nt + 1;
    std::vector<double> Gt((size_t)mt * mt);

    // JTJ (np x np), g = J^T r (np) and the cost at p; P at p in Pj
    std::vector<double> JTJ((size_t)np * np), g(np), Pj;
    auto eval = [&](const ThetaParam& t, const double* pp, std::vector<double>& jtj, std::vector<double>& gg,
                    std::vector<double>& Pm, double& cst) -> ftsp2_status {
        if (launch_train_fwd_jac(target, beta0, mu0, L, alpha, t, dX, nsamples, dRr, dM, s, fam) != cudaSuccess)
            return FTSP2_E_CUDA;
        if (launch_train_gram(dM, nsamples, nt, dG, dPart, tl.nchunks, s) != cudaSuccess) return FTSP2_E_CUDA;
        if (cudaMemcpyAsync(Gt.data(), dG, sizeof(double) * mt * mt, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return FTSP2_E_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return FTSP2_E_CUDA;
        form_jacobian(form, L, pp, Pm, fd);
        cst = 0.5 * Gt[(size_t)nt * mt + nt];
        std::vector<double> GP((size_t)nt * np, 0.0);   // (J^T J) P
        for (int i = 0; i < nt; ++i)
            for (int k = 0; k < nt; ++k) {
                const double v = Gt[(size_t)i * mt + k];
                if (v == 0.0) continue;
                for (int j = 0; j < np; ++j) GP[(size_t)i * np + j] += v * Pm[(size_t)k * np + j];
            }
        jtj.assign((size_t)np * np, 0.0);
        gg.assign(np, 0.0);
        for (int k = 0; k < nt; ++k)
            for (int i = 0; i < np; ++i) {
                const double pk = Pm[(size_t)k * np + i];
                if (pk == 0.0) continue;
                for (int j = 0; j < np; ++j) jtj[(size_t)i * np + j] += pk * GP[(size_t)k * np + j];
                gg[i] += pk * Gt[(size_t)k * mt + nt];
            }
        return FTSP2_OK;
    };

    double cost = 0.0;
    st = eval(tp, p.data(), JTJ, g, Pj, cost);
    if (st != FTSP2_OK) return st;
    const double cost0 = cost;
    double lam = 1e-3;
    int accepted = 0, it = 0;
    const double h = 0.1;
    std::vector<double> Md((size_t)np * np), v, a, rhs(np), JTJc, gc, Pc, vt(nt);
    for (it = 0; it < iterations; ++it) {
        Md = JTJ;
        // FORM_SKIPK: a zero diagonal entry (a parameter the output does not
        // depend on at p, e.g. the feedback of an accumulator that is still
        // zero) is damped with the smallest positive one, so Md stays regular
        double dmin = 0.0;
        if (form == FORM_SKIPK)
            for (int i = 0; i < np; ++i) {
                const double dv = JTJ[(size_t)i * np + i];
                if (dv > 0.0 && (dmin == 0.0 || dv < dmin)) dmin = dv;
            }
        for (int i = 0; i < np; ++i) {
            const double dv = JTJ[(size_t)i * np + i];
            Md[(size_t)i * np + i] += lam * (form == FORM_SKIPK && dv <= 0.0 ? (dmin > 0.0 ? dmin : 1.0) : dv);
        }
        for (int i = 0; i < np; ++i) rhs[i] = -g[i];
        if (!chol_solve(Md, np, rhs, v)) {
            lam = std::min(lam * 10.0, 1e12);
            continue;
        }
        std::vector<double> step = v;
        if (accel) {
            // second directional derivative of r along p + tau v, by finite
            // differences at tau = h, with J v = J (P v) from the stored Jacobian
            std::vector<double> ph(p);
            for (int i = 0; i < np; ++i) ph[i] += h * v[i];
            ThetaParam th_h;
            if (form_theta(form, L, ph.data(), th_h, fd) != FTSP2_OK) return FTSP2_E_ARG;
            for (int k = 0; k < nt; ++k) {
                double acc = 0.0;
                for (int j = 0; j < np; ++j) acc += Pj[(size_t)k * np + j] * v[j];
                vt[k] = acc;
            }
            std::vector<double> rt(nt);
            if (launch_train_residual(target, beta0, mu0, L, alpha, th_h, dX, nsamples, dRh, s, fam) != cudaSuccess ||
                cudaMemcpyAsync(dV, vt.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                launch_train_accel(dM, dV, dRh, h, nsamples, nt, dAp, dOut, s) != cudaSuccess ||
                cudaMemcpyAsync(rt.data(), dOut, sizeof(double) * nt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return FTSP2_E_CUDA;
            for (int i = 0; i < np; ++i) {
                double acc = 0.0;
                for (int k = 0; k < nt; ++k) acc += Pj[(size_t)k * np + i] * rt[k];
                rhs[i] = -acc;
            }
            if (chol_solve(Md, np, rhs, a)) {
                double na = 0, nv = 0;
                for (int i = 0; i < np; ++i) {
                    na += a[i] * a[i];
                    nv += v[i] * v[i];
                }
                if (2.0 * std::sqrt(na) <= 0.75 * std::sqrt(nv))
                    for (int i = 0; i < np; ++i) step[i] = v[i] + 0.5 * a[i];
            }
        }
        std::vector<double> pc(p);
        for (int i = 0; i < np; ++i) pc[i] += step[i];
        ThetaParam cand;
        double cc = INFINITY;
        if (form_theta(form, L, pc.data(), cand, fd) == FTSP2_OK) {
            st = eval(cand, pc.data(), JTJc, gc, Pc, cc);
            if (st != FTSP2_OK) return st;
        }
        if (std::isfinite(cc) && cc < cost) {
            p.swap(pc);
            tp = cand;
            JTJ.swap(JTJc);
            g.swap(gc);
            Pj.swap(Pc);
            cost = cc;
            lam = std::max(lam / 10.0, 1e-12);
            ++accepted;
        } else {
            lam = std::min(lam * 10.0, 1e12);
        }
    }
    // residuals at the final table and their max
    if (launch_train_residual(target, beta0, mu0, L, alpha, tp, dX, nsamples, dRr, s, fam) != cudaSuccess ||
        launch_train_absmax(dRr, nsamples, dAm + 8, dAm, s) != cudaSuccess)
        return FTSP2_E_CUDA;
    double mx = 0;
    if (cudaMemcpyAsync(&mx, dAm, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FTSP2_E_CUDA;
    for (int i = 0; i < np; ++i) p_out[i] = p[i];
    if (rep) {
        rep->iterations = it;
        rep->accepted = accepted;
        rep->cost0 = cost0;
        rep->cost = cost;
        rep->max_err = mx;
        rep->lambda = lam;
    }
    return FTSP2_OK;
}

// The sample set (built on the host, copied into the workspace) and the
// default start of each form, then the LM fit on the device.
// Default start of a FORM_SKIPK fit: the one-accumulator embedding of the
// Eq. mlsp2 start (ftsp2_mlsp2_to_skip), its connections in slots 0 and its
// constant in slot k; the further stored layers and accumulator inputs gamma
// zero, the further accumulators' feedback beta kSkipkBetaStart (no effect
// while those accumulators are zero; nonzero, so that their gamma have a
// derivative and the fit can open them).
constexpr double kSkipkBetaStart = 0.01;

static void skipk_start(int L, const FormDims& fd, double beta0, double mu0, double* p) {
    const int k = fd.k, K = fd.K;
    std::vector<double> th(4 * L), tab(4 * L + 4);
    train_init_mlsp2(L, beta0, mu0, th.data());
    mlsp2_to_skip(L, th.data(), tab.data());
    double* al = p;
    double* be = al + L * (k + 1);
    double* ga = be + L * K;
    std::fill(p, p + form_params(FORM_SKIPK, L, fd), 0.0);
    for (int i = 0; i < L; ++i) {
        al[i * (k + 1) + 0] = tab[4 * i + 1];
        al[i * (k + 1) + k] = tab[4 * i + 0];
        for (int l = 0; l < K; ++l) {
            be[i * K + l] = l == 0 ? tab[4 * i + 2] : kSkipkBetaStart;
            ga[i * K + l] = l == 0 ? tab[4 * i + 3] : 0.0;
        }
    }
    ga[L * K] = tab[4 * L];          // A_{0,1}
    ga[L * K + 1] = tab[4 * L + 1];  // gamma_L
}

static ftsp2_status train_entry(int form, int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                uint64_t seed, int iterations, int accel, const double* p_init, double* p_out,
                                ftsp2_train_report* rep, void* dWork, size_t work_bytes, void* stream,
                                const FormDims& fd = FormDims()) {
    if (nsamples < 1 || !dWork || !p_out || !(beta0 > 0.0) || !(mu0 > 0.0 && mu0 < 1.0)) return FTSP2_E_ARG;
    const bool maxf = form == FORM_MAX || form == FORM_SKIPK;
    if (L < 1 || L > (form == FORM_SKIP ? kMaxLayers - 1 : maxf ? kMaxMaxLayers : kMaxLayers)) return FTSP2_E_ARG;
    if (form == FORM_SKIPK && (fd.k < 1 || fd.K < 1 || fd.k > L)) return FTSP2_E_ARG;
    const TrainLayout tl = train_layout(nsamples, form_layout_rows(form, L));
    if (work_bytes < tl.total) return FTSP2_E_WORKSPACE;
    std::vector<double> x((size_t)nsamples);
    train_sample_grid(beta0, mu0, nsamples, seed, x.data());
    double* dX = reinterpret_cast<double*>(static_cast<uint8_t*>(dWork) + tl.X);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(dX, x.data(), sizeof(double) * nsamples, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FTSP2_E_CUDA;
    std::vector<double> init;
    if (!p_init) {
        if (form == FORM_MLSP2) {
            init.resize(4 * L);
            train_init_mlsp2(L, beta0, mu0, init.data());
        } else if (form == FORM_ALT) {
            init.resize(2 * L + 2);
            train_init_alt(L, mu0, init.data());
        } else if (form == FORM_MAX) {
            std::vector<double> th(4 * L);
            train_init_mlsp2(L, beta0, mu0, th.data());
            init.resize(max_nparams(L));
            const ftsp2_status st = ftsp2_mlsp2_to_max(L, th.data(), init.data());
            if (st != FTSP2_OK) return st;
        } else if (form == FORM_SKIPK) {
            init.resize(form_params(FORM_SKIPK, L, fd));
            skipk_start(L, fd, beta0, mu0, init.data());
        } else {
            std::vector<double> th(4 * L);
            train_init_mlsp2(L, beta0, mu0, th.data());
            init.resize(4 * L + 4);
            mlsp2_to_skip(L, th.data(), init.data());
        }
        p_init = init.data();
    }
    if (form != FORM_SKIP)
        return lm_train(form, target, beta0, mu0, L, alpha, dX, nsamples, iterations, accel, p_init, p_out, rep,
                        dWork, work_bytes, stream, fd);
    // the table's (L + 1) x 4 rows: the output row's last two entries are unused
    std::vector<double> p(4 * L + 2), out(4 * L + 2);
    std::copy(p_init, p_init + 4 * L + 2, p.begin());
    const ftsp2_status st = lm_train(FORM_SKIP, target, beta0, mu0, L, alpha, dX, nsamples, iterations, accel,
                                     p.data(), out.data(), rep, dWork, work_bytes, stream);
    if (st != FTSP2_OK) return st;
    std::copy(out.begin(), out.end(), p_out);
    p_out[4 * L + 2] = p_out[4 * L + 3] = 0.0;
    return FTSP2_OK;
}

ftsp2_status ftsp2_train_coeffs(int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                uint64_t seed, int iterations, int accel, const double* theta_init,
                                double* theta_out, ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                void* stream) {
    return train_entry(FORM_MLSP2, target, beta0, mu0, L, alpha, nsamples, seed, iterations, accel, theta_init,
                       theta_out, rep, dWork, work_bytes, stream);
}

ftsp2_status ftsp2_train_coeffs_alt(int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                    uint64_t seed, int iterations, int accel, const double* alt_init,
                                    double* alt_out, ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                    void* stream) {
    return train_entry(FORM_ALT, target, beta0, mu0, L, alpha, nsamples, seed, iterations, accel, alt_init, alt_out,
                       rep, dWork, work_bytes, stream);
}

ftsp2_status ftsp2_train_coeffs_skip(int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                     uint64_t seed, int iterations, int accel, const double* skip_init,
                                     double* skip_out, ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                     void* stream) {
    return train_entry(FORM_SKIP, target, beta0, mu0, L, alpha, nsamples, seed, iterations, accel, skip_init,
                       skip_out, rep, dWork, work_bytes, stream);
}

size_t ftsp2_train_workspace_size_max(int nsamples, int L) {
    if (nsamples < 1 || L < 1 || L > kMaxMaxLayers) return 0;
    return train_layout(nsamples, form_layout_rows(FORM_MAX, L)).total;
}

ftsp2_status ftsp2_train_coeffs_max(int target, double beta0, double mu0, int L, double alpha, int nsamples,
                                    uint64_t seed, int iterations, int accel, const double* max_init, double* max_out,
                                    ftsp2_train_report* rep, void* dWork, size_t work_bytes, void* stream) {
    return train_entry(FORM_MAX, target, beta0, mu0, L, alpha, nsamples, seed, iterations, accel, max_init, max_out,
                       rep, dWork, work_bytes, stream);
}

ftsp2_status ftsp2_train_coeffs_skipk(int target, double beta0, double mu0, int L, int k, int K, double alpha,
                                      int nsamples, uint64_t seed, int iterations, int accel, const double* skip_init,
                                      double* skip_out, ftsp2_train_report* rep, void* dWork, size_t work_bytes,
                                      void* stream) {
    FormDims fd;
    fd.k = k;
    fd.K = K;
    return train_entry(FORM_SKIPK, target, beta0, mu0, L, alpha, nsamples, seed, iterations, accel, skip_init,
                       skip_out, rep, dWork, work_bytes, stream, fd);
}

ftsp2_status ftsp2_train_init_skipk(int L, int k, int K, double beta0, double mu0, double* skip_out) {
    if (L < 1 || L > kMaxMaxLayers || k < 1 || K < 1 || k > L || !skip_out || !(beta0 > 0.0) ||
        !(mu0 > 0.0 && mu0 < 1.0))
        return FTSP2_E_ARG;
    FormDims fd;
    fd.k = k;
    fd.K = K;
    skipk_start(L, fd, beta0, mu0, skip_out);
    return FTSP2_OK;
}

ftsp2_status ftsp2_skipk_to_max(int L, int k, int K, const double* skip, double* max_out) {
    if (L < 1 || L > kMaxMaxLayers || k < 1 || K < 1 || !skip || !max_out) return FTSP2_E_ARG;
    FormDims fd;
    fd.k = k;
    fd.K = K;
    return skipk_theta(L, fd, skip, max_out);
}

ftsp2_status ftsp2_skip_to_max(int L, int k, int K, const double* alpha, const double* beta, const double* gamma,
                               const double* A0, double gamma_L, double* max_out) {
    if (L < 1 || L > kMaxMaxLayers || k < 1 || K < 0 || !alpha || !max_out || (K > 0 && (!beta || !gamma || !A0)) ||
        !std::isfinite(gamma_L))
        return FTSP2_E_ARG;
    for (int i = 0; i < L * (k + 1); ++i)
        if (!std::isfinite(alpha[i])) return FTSP2_E_ARG;
    for (int i = 0; i < L * K; ++i)
        if (!std::isfinite(beta[i]) || !std::isfinite(gamma[i])) return FTSP2_E_ARG;
    for (int l = 0; l < K; ++l)
        if (!std::isfinite(A0[l])) return FTSP2_E_ARG;
    int o = 0;
    for (int i = 0; i < L; ++i) {
        double dl = alpha[i * (k + 1) + k];
        for (int l = 0; l < K; ++l) dl += beta[i * K + l] * A0[l];
        max_out[o] = dl;
        double gs = 0.0;
        for (int l = 0; l < K; ++l) gs += gamma[i * K + l];
        max_out[o + 1] = gs;
        for (int j = 0; j <= i; ++j) {
            double th = 0.0;
            if (j < i)
                for (int l = 0; l < K; ++l) th += beta[i * K + l] * gamma[j * K + l];
            if (i - j < k) th += alpha[i * (k + 1) + (i - j)];
            max_out[o + 2 + j] = th;
        }
        o += i + 3;
    }
    double c = 0.0;
    for (int l = 0; l < K; ++l) c += A0[l];
    max_out[o] = c;
    max_out[o + 1] = gamma_L;
    return FTSP2_OK;
}

ftsp2_status ftsp2_mlsp2_to_max(int L, const double* theta, double* max_out) {
    if (L < 1 || L > kMaxMaxLayers || !theta || !max_out) return FTSP2_E_ARG;
    std::vector<double> sk(4 * (L + 1));
    const ftsp2_status st = ftsp2_mlsp2_to_skip(L, theta, sk.data());
    if (st != FTSP2_OK) return st;
    // Skip-SP2 rows (delta, alpha, beta, gamma) with output row (A_0, gamma_L):
    // u_i = delta_i + alpha_i x_i + beta_i (A_0 + sum_{j<i} gamma_j x_j)
    int o = 0;
    const double A0 = sk[4 * L], gL = sk[4 * L + 1];
    for (int i = 0; i < L; ++i) {
        max_out[o] = sk[4 * i] + sk[4 * i + 2] * A0;
        max_out[o + 1] = sk[4 * i + 3];
        for (int j = 0; j < i; ++j) max_out[o + 2 + j] = sk[4 * i + 2] * sk[4 * j + 3];
        max_out[o + 2 + i] = sk[4 * i + 1];
        o += i + 3;
    }
    max_out[o] = A0;
    max_out[o + 1] = gL;
    return FTSP2_OK;
}

ftsp2_status ftsp2_train_residuals(int family, int target, double beta0, double mu0, int L, double alpha,
                                   const double* table, const double* dX, int npoints, double* dR, void* stream) {
    if ((target != FTSP2_TARGET_FERMI && target != FTSP2_TARGET_ENTROPY) || !table || !dX || !dR || npoints < 1)
        return FTSP2_E_ARG;
    if (family != FTSP2_FAMILY_MLSP2 && family != FTSP2_FAMILY_SKIP && family != FTSP2_FAMILY_MAX)
        return FTSP2_E_ARG;
    if (L < 1 || L > (family == FTSP2_FAMILY_SKIP  ? kMaxLayers - 1
                      : family == FTSP2_FAMILY_MAX ? kMaxMaxLayers
                                                   : kMaxLayers))
        return FTSP2_E_ARG;
    const int nv = family == FTSP2_FAMILY_SKIP ? 4 * L + 2 : family == FTSP2_FAMILY_MAX ? max_nparams(L) : 4 * L;
    ThetaParam tp;
    std::memset(&tp, 0, sizeof(tp));
    for (int i = 0; i < nv; ++i) {
        if (!std::isfinite(table[i])) return FTSP2_E_ARG;
        tp.v[i] = table[i];
    }
    return from_cuda(launch_train_residual(target, beta0, mu0, L, alpha, tp, dX, npoints, dR,
                                           static_cast<cudaStream_t>(stream), family));
}

ftsp2_status ftsp2_train_samples(double beta0, double mu0, int nsamples, uint64_t seed, double* x_out) {
    if (nsamples < 1 || !x_out || !(beta0 > 0.0) || !(mu0 > 0.0 && mu0 < 1.0)) return FTSP2_E_ARG;
    train_sample_grid(beta0, mu0, nsamples, seed, x_out);
    return FTSP2_OK;
}

ftsp2_status ftsp2_train_init(int L, double beta0, double mu0, double* theta_out) {
    if (L < 1 || L > kMaxLayers || !theta_out || !(beta0 > 0.0) || !(mu0 > 0.0 && mu0 < 1.0)) return FTSP2_E_ARG;
    train_init_mlsp2(L, beta0, mu0, theta_out);
    return FTSP2_OK;
}

ftsp2_status ftsp2_train_init_alt(int L, double mu0, double* alt_out) {
    if (L < 1 || L > kMaxLayers || !alt_out || !(mu0 > 0.0 && mu0 < 1.0)) return FTSP2_E_ARG;
    train_init_alt(L, mu0, alt_out);
    return FTSP2_OK;
}

ftsp2_status ftsp2_mlsp2_to_skip(int L, const double* theta, double* skip_out) {
    if (L < 1 || L > kMaxLayers - 1 || !theta || !skip_out) return FTSP2_E_ARG;
    for (int i = 0; i < 4 * L; ++i)
        if (!std::isfinite(theta[i])) return FTSP2_E_ARG;
    for (int i = 0; i < L; ++i)
        if (theta[4 * i] == 0.0) return FTSP2_E_ARG;        // a linear layer has no square form
    mlsp2_to_skip(L, theta, skip_out);
    return FTSP2_OK;
}

double ftsp2_layer_count(double beta_p) {
    // Eq. layer count: n_l = ln(beta'/4) / ln(2 phi), phi = 1/varphi (Sec. IV B)
    if (!(beta_p > 0.0)) return NAN;
    const double phi = 2.0 / (1.0 + std::sqrt(5.0));
    return std::log(beta_p / 4.0) / std::log(2.0 * phi);
}

ftsp2_status ftsp2_alt_to_mlsp2(int L, const double* alt, double* theta_out) {
    if (!alt || !theta_out || L < 1 || L > kMaxLayers) return FTSP2_E_ARG;
    for (int i = 0; i < 2 * L + 2; ++i)
        if (!std::isfinite(alt[i])) return FTSP2_E_ARG;
    alt_rows(L, alt, theta_out);
    return FTSP2_OK;
}

}  // extern "C"
