// (a3)-(a6) One layer of the learned recursion (Eq. mlsp2) for every active
// (instance, chain) of a grouped launch, on the 5th-generation tensor cores.
//
// The product of a layer is the symmetric square Z^2 of the centred state.
// Only output tiles that touch the upper triangle are computed; each element
// (r, c) with r <= c is produced once and written to (r, c) and (c, r).  Since
// Z is symmetric, (Z^2)_{rc} = sum_k Z_{rk} Z_{ck}: both MMA operands are
// K-major row panels of the same matrix, loaded by TMA with 128-byte swizzle.
//
// Split precision (Sec. IV A, Eq. emulated matmul, generalised): Z is stored as
// NSPLIT low-precision planes Z = sum_s Z_s and the products Z_s Z_t with
// s + t small enough are accumulated into one FP32 TMEM accumulator:
//   FP16X2: (0,0) (0,1) (1,0)    TF32X3: same      BF16X3: + (0,2) (2,0) (1,1)
// (the paper's two GEMMs plus a transpose-add become three products on the
// triangle, which costs 1.5 n^3 MACs instead of 2 n^3).
//
// Warp roles (192 threads, one CTA per SM, persistent over the tile list):
//   warp 0 lane 0: TMA producer (STAGES-deep ring of K-slices)
//   warp 1 lane 0: tcgen05.mma issuer; warp 1 also allocates TMEM
//   warps 2-5    : epilogue, one 32-lane TMEM quarter each, double-buffered
//                  accumulators so the epilogue of tile t overlaps the MMAs of
//                  tile t+1.
// Every wait is bounded (ftsp2::mbar_wait): on timeout the CTA sets
// FTSP2_E_TIMEOUT in the status word and all roles leave their loops.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "epilogue.cuh"
#include "ftsp2_internal.h"

namespace ftsp2 {

template <int MODE>
struct TcCfg;

template <>
struct TcCfg<FTSP2_FP16X2> {
    static constexpr int NSPLIT = 2, ESIZE = 2, BKE = 64, BN = 256, STAGES = 2, NPROD = 3;
    static constexpr uint32_t ATYPE = 0;      // f16
    static constexpr bool TF32 = false;
};
template <>
struct TcCfg<FTSP2_BF16X3> {
    static constexpr int NSPLIT = 3, ESIZE = 2, BKE = 64, BN = 128, STAGES = 2, NPROD = 6;
    static constexpr uint32_t ATYPE = 1;      // bf16
    static constexpr bool TF32 = false;
};
template <>
struct TcCfg<FTSP2_TF32X3> {
    static constexpr int NSPLIT = 2, ESIZE = 4, BKE = 32, BN = 256, STAGES = 2, NPROD = 3;
    static constexpr uint32_t ATYPE = 2;      // tf32
    static constexpr bool TF32 = true;
};

__device__ __constant__ int kProdA[6] = {0, 0, 1, 0, 2, 1};
__device__ __constant__ int kProdB[6] = {0, 1, 0, 2, 0, 1};

// Instruction descriptor of tcgen05.mma kind::f16 / kind::tf32: D in FP32,
// A and B K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t atype, int M, int N) {
    return (1u << 4)                       // D format: F32
           | (atype << 7) | (atype << 10)  // A, B formats
           | ((uint32_t)(N >> 3) << 17)    // N >> 3
           | ((uint32_t)(M >> 4) << 24);   // M >> 4
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128 bytes,
// 8-row swizzle atoms of 1024 bytes (stride byte offset), version bits 46-48 = 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                     uint32_t accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ----------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(192, 1)
    layer_tc_kernel(const __grid_constant__ LayerArgs a, const __grid_constant__ TmaMaps maps) {
    using C = TcCfg<MODE>;
    constexpr int BN = C::BN;
    constexpr int A_PLANE = kTileM * 128;
    constexpr int B_PLANE = BN * 128;
    constexpr int STAGE_BYTES = C::NSPLIT * (A_PLANE + B_PLANE);
    constexpr int KSTEPS = 4;                 // 128-byte slice / 32 bytes per MMA
    constexpr uint32_t IDESC = make_idesc(C::ATYPE, kTileM, BN);
    constexpr uint32_t TMEM_COLS = 2 * BN;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[C::STAGES];
    __shared__ __align__(8) uint64_t empty_bar[C::STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];
    __shared__ __align__(8) uint64_t tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull_bar[s], 1);
            mbar_init(&tempty_bar[s], 4);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            for (int t = blockIdx.x; t < a.ntiles && !abort_flag; t += gridDim.x) {
                const Tile tl = a.tiles[t];
                int k;
                if (!tile_active(a, tl, k)) continue;
                const int n = a.inst[tl.inst].n;
                const int nk = (n + C::BKE - 1) / C::BKE;
                const int rowA = tl.inst * a.P + tl.I * kTileM;
                const int rowB = tl.inst * a.P + tl.J * BN;
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[stage]);
                    mbar_expect_tx(&full_bar[stage], STAGE_BYTES);
                    uint8_t* sbase = smem + stage * STAGE_BYTES;
#pragma unroll
                    for (int s = 0; s < C::NSPLIT; ++s) {
                        tma_load_2d(smem_u32(sbase + s * A_PLANE), &maps.a[tl.chain][s], fb, kb * C::BKE, rowA);
                        tma_load_2d(smem_u32(sbase + C::NSPLIT * A_PLANE + s * B_PLANE), &maps.b[tl.chain][s], fb,
                                    kb * C::BKE, rowB);
                    }
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t aphase = 0;
            for (int t = blockIdx.x; t < a.ntiles && !abort_flag; t += gridDim.x) {
                const Tile tl = a.tiles[t];
                int k;
                if (!tile_active(a, tl, k)) continue;
                const int n = a.inst[tl.inst].n;
                const int nk = (n + C::BKE - 1) / C::BKE;
                if (!mbar_wait(&tempty_bar[buf], aphase ^ 1u, &abort_flag, a.status)) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&full_bar[stage], phase, &abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < KSTEPS; ++kk) {
#pragma unroll
                        for (int p = 0; p < C::NPROD; ++p) {
                            const uint32_t sa = sb + kProdA[p] * A_PLANE + kk * 32;
                            const uint32_t sbb = sb + C::NSPLIT * A_PLANE + kProdB[p] * B_PLANE + kk * 32;
                            umma<C::TF32>(dt, sdesc_sw128(sa), sdesc_sw128(sbb), IDESC,
                                          (kb | kk | p) != 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(smem_u32(&empty_bar[stage]));
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                umma_commit(smem_u32(&tfull_bar[buf]));
                if (++buf == 2) {
                    buf = 0;
                    aphase ^= 1u;
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;                // TMEM lane quarter of this warp
        int buf = 0;
        uint32_t aphase = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            const Tile tl = a.tiles[t];
            int k;
            if (!tile_active(a, tl, k)) continue;
            if (!mbar_wait(&tfull_bar[buf], aphase, &abort_flag, a.status)) break;
            tc_fence_after();
            EpiCtx e;
            make_ctx(a, tl, k, e, MODE == FTSP2_FP16X2);
            const int r = tl.I * kTileM + q * 32 + lane;
            const int rmin = tl.I * kTileM + q * 32;
            double tr = 0.0, sq = 0.0;
            for (int cc = 0; cc < BN / 16; ++cc) {
                const int c0 = tl.J * BN + cc * 16;
                if (c0 >= e.n) break;                 // warp-uniform
                if (c0 + 15 < rmin) continue;         // whole chunk below the diagonal
                if (rmin >= e.n) break;
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + cc * 16), v);
                epi_segment<16>(a, e, r, c0, v, tr, sq);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty_bar[buf]);
            if (a.last) {
                for (int o = 16; o > 0; o >>= 1) {
                    tr += __shfl_xor_sync(0xffffffffu, tr, o);
                    sq += __shfl_xor_sync(0xffffffffu, sq, o);
                }
                if (lane == 0) {
                    a.partials[((size_t)t * 4 + q) * 2 + 0] = tr;
                    a.partials[((size_t)t * 4 + q) * 2 + 1] = sq;
                }
            }
            if (++buf == 2) {
                buf = 0;
                aphase ^= 1u;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

int tc_block_n(int mode) {
    switch (mode) {
        case FTSP2_FP16X2: return TcCfg<FTSP2_FP16X2>::BN;
        case FTSP2_BF16X3: return TcCfg<FTSP2_BF16X3>::BN;
        case FTSP2_TF32X3: return TcCfg<FTSP2_TF32X3>::BN;
    }
    return 0;
}

template <int MODE>
static int smem_of() {
    using C = TcCfg<MODE>;
    return C::STAGES * C::NSPLIT * (kTileM * 128 + C::BN * 128) + 1024;
}

int tc_smem_bytes(int mode) {
    switch (mode) {
        case FTSP2_FP16X2: return smem_of<FTSP2_FP16X2>();
        case FTSP2_BF16X3: return smem_of<FTSP2_BF16X3>();
        case FTSP2_TF32X3: return smem_of<FTSP2_TF32X3>();
    }
    return 0;
}

template <int MODE>
static cudaError_t launch_mode(const LayerArgs& a, const TmaMaps& maps, int grid, cudaStream_t s) {
    const int smem = smem_of<MODE>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(layer_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    layer_tc_kernel<MODE><<<grid, 192, smem, s>>>(a, maps);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_layer_tc(int mode, const LayerArgs& a, const TmaMaps& maps, int grid, cudaStream_t s) {
    switch (mode) {
        case FTSP2_FP16X2: return launch_mode<FTSP2_FP16X2>(a, maps, grid, s);
        case FTSP2_BF16X3: return launch_mode<FTSP2_BF16X3>(a, maps, grid, s);
        case FTSP2_TF32X3: return launch_mode<FTSP2_TF32X3>(a, maps, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ftsp2
