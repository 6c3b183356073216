// (a3)-(a6) Layers of the learned recursion (Eq. mlsp2) for every active
// (instance, chain) of a grouped launch, on the 5th-generation tensor cores:
// one layer per launch, or consecutive layers of the main format in one
// persistent cooperative launch (below).
//
// The product of a layer is the symmetric square Z^2 of the centred state.
// Output tiles are square (256 x 256 on CTA pairs or 128 x 128 on single CTAs,
// chosen per call) and only those touching the upper triangle are computed
// (I <= J); each element (r, c) with r <= c is produced once.  Since Z is
// symmetric, (Z^2)_{rc} = sum_k Z_{rk} Z_{ck}: both MMA operands are row
// panels of the same matrix, loaded by TMA with 128-byte swizzle.  The next
// operands are stored for the upper triangle plus the diagonal tile blocks
// (the mirror (c, r) everywhere only before a layer that reads full
// matrices); K-slices left of a panel's diagonal block are loaded as
// transposed 64 x 64 panels of the upper triangle (MN-major operands).
//
// Split precision (Sec. IV A, Eq. emulated matmul, generalised): Z is stored as
// NSPLIT low-precision planes Z = sum_s Z_s and the products Z_s Z_t with
// s + t small enough are accumulated in FP32:
//   FP16X2: (0,0) (0,1) (1,0)    TF32X3: same      BF16X3: + (0,2) (2,0) (1,1)
// (the paper's two GEMMs plus a transpose-add become three products on the
// triangle: 1.5 n^3 MACs instead of 2 n^3).
//
// CTA pairs (cta_group::2).  A cluster of two CTAs computes one 256 x 256 tile
// with M = 256 MMAs issued by the even CTA: CTA r loads its own 128 rows of
// the A panel and its 128-row half of the B panel, so each SM fills and reads
// half of B.  Both CTAs' TMA loads complete on the even CTA's "full" barrier;
// the MMA commit is multicast to both CTAs' "empty" and "tfull" barriers; the
// odd CTA's epilogue warps release accumulators on the even CTA's "tempty".
// Single CTAs (cta_group::1) run the same pipeline on 128 x 128 tiles with
// M = 128 MMAs: a quarter of the padding of a pair tile on the diagonal and at
// ragged edges, which pays for batches of small instances.
//
// Chunked accumulation.  Every 128 elements of K (CK slices; a launch may ask
// for shorter chunks) the MMAs switch to the next of the TMEM chunk
// accumulators (two on a CTA pair, four on a single CTA) and the epilogue adds
// the finished chunk into FP32 registers; the tensor core's internal
// accumulation then spans 128 products per chunk instead of all n.  Measured at n = 4096 with the
// printed table (density, FP16X2): chunks of 256 / 128 / 64 elements give
// max|D - D_ref| = 1.85e-6 / 9.0e-7 / 6.9e-7 at layer times 0.235 / 0.251 /
// 0.314 ms; 128 is the default.
//
// Warp roles (576 threads per CTA, 640 with the deferred epilogue; persistent
// over the tile list):
//   warp 0 lane 0 : TMA producer (STAGES-deep ring of 128-byte K-slices)
//   warp 1        : TMEM allocation; lane 0 of the even CTA issues tcgen05.mma
//   warps 2..17   : accumulating warps; warp w reads TMEM lane quarter w % 4
//                   and column quarter (w - 2) / 4 of the CTA's 128-row
//                   accumulator and adds the chunks in FP32 registers
//   warps 18..19  : (deferred epilogue only) store warps.
// Final epilogue of a tile (Z_{k+1}, A_{k+1}, next operands).  Inline: the
// accumulating warps write the finished sum back into the last chunk's TMEM
// buffer and run the epilogue from there while the MMAs of the next tile fill
// the other buffer (one chunk ahead).  Deferred (pair tiles, long K): they
// store the sum to a per-CTA scratch in global memory and go on with the next
// tile at once; the two store warps stream scratch, Z_k and A_k through a small
// shared ring (cp.async) and write the results while the next tile's MMAs run.
// A unit's last tile always runs inline, so no store-warp tail follows the
// last MMAs.
// Multi-layer launches (a.nlayers > 1).  The work items are (layer, tile) in
// layer order; every role walks the same item sequence.  An item of layer g
// waits (producer) until all tiles of layer g - 1 of its instance and chain
// have finished their epilogues: each CTA counts kEpiWarps completions per tile
// in the instance's counter (accumulating warps 1 each, store warps
// kEpiWarps / kStoreWarps each, the producer kEpiWarps for an inactive item),
// released by a fence before the atomic and acquired by the readers, with a
// proxy fence before the TMA loads of the new operands.  Dependencies point
// only to earlier items and a unit takes its items in order, so the waits end;
// the CTAs of such a launch are co-resident (cooperative launch).
// Every wait is bounded (a.wait_ns).  A dependency wait that runs out records
// FTSP2_E_TIMEOUT in the status word of the call; from then on every role of
// every CTA that sees the failure runs the rest of its work items in skip
// mode: the same barrier arrivals, waits and commits in the same order, but no
// TMA loads, MMAs or epilogue stores.  Every barrier phase therefore still
// completes and nothing is in flight when the work list ends; the MMA issuer
// also waits for a last commit of its own before the CTAs free TMEM.  A
// pipeline wait that runs out twice (a broken protocol, not expected) leaves
// its loop after a bounded grace period for the copies in flight.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "epilogue.cuh"
#include "ftsp2_internal.h"

namespace ftsp2 {

template <int MODE>
struct TcCfg;

template <>
struct TcCfg<FTSP2_FP16X2> {
    static constexpr int NSPLIT = 2, ESIZE = 2, STAGES = 3, NPROD = 3, CK = 2;
    static constexpr uint32_t ATYPE = 0;      // f16
    static constexpr bool TF32 = false;
};
template <>
struct TcCfg<FTSP2_BF16X3> {
    static constexpr int NSPLIT = 3, ESIZE = 2, STAGES = 2, NPROD = 6, CK = 2;
    static constexpr uint32_t ATYPE = 1;      // bf16
    static constexpr bool TF32 = false;
};
template <>
struct TcCfg<FTSP2_TF32X3> {
    static constexpr int NSPLIT = 2, ESIZE = 4, STAGES = 3, NPROD = 3, CK = 4;
    static constexpr uint32_t ATYPE = 2;      // tf32
    static constexpr bool TF32 = true;
};

// Tile geometry.  PAIR = true: clusters of two CTAs, 256 x 256 tiles, M = 256
// MMAs (the default for large matrices).  PAIR = false: one CTA, 128 x 128
// tiles, M = 128 MMAs (less padding for small instances of a ragged batch).
template <bool PAIR>
struct Geo {
    static constexpr int TILE = PAIR ? 256 : 128;    // rows = columns of a tile
    static constexpr int NCTA = PAIR ? 2 : 1;
    // TMEM chunk accumulators (512 columns): two of 256 columns on a pair,
    // four of 128 on a single CTA, so that the MMAs of the next tile can run
    // three chunks ahead of a single CTA's final epilogue
    static constexpr int NBUF = PAIR ? 2 : 4;
};
constexpr int kCtaRows = 128;
constexpr int kEpiWarps = 16;
constexpr int kGrp = 8;                            // columns per epilogue group
// Deferred final epilogue: store warps, their shared-memory staging ring
// (entries of 16 columns x 32 rows: sums, Z_k, A_k) and the per-CTA scratch
// of finished tile sums in global memory (one 32-row x 64-column block per
// accumulating warp, in the blocked layout of the state).
constexpr int kStoreWarps = 2;
constexpr int kRing = 2;
constexpr int kEntryBytes = 3 * 2048;
constexpr int kItemFloats = 2048;
static_assert(kEpiWarps * kItemFloats == kEpiScratchFloats, "scratch of one CTA");
// multi-layer launches: the store warps' shares of a tile's completions add up
// to the kEpiWarps that the accumulating warps give for an inline tile
static_assert(kEpiWarps % kStoreWarps == 0, "completion shares of the store warps");
__host__ __device__ constexpr int threads_of(bool deferred) {
    return 64 + 32 * (kEpiWarps + (deferred ? kStoreWarps : 0));
}
static_assert(kPartialSlots == 2 * kEpiWarps, "one partial-sum slot per epilogue warp of the pair");

// split planes (s, t) of the products Z_s Z_t, in issue order
__host__ __device__ constexpr int prod_a(int p) { return p == 2 ? 1 : (p == 4 ? 2 : (p == 5 ? 1 : 0)); }
__host__ __device__ constexpr int prod_b(int p) { return p == 1 ? 1 : (p == 3 ? 2 : (p == 5 ? 1 : 0)); }

// Instruction descriptor of tcgen05.mma kind::f16 / kind::tf32: D in FP32,
// A and B K-major, M x N.
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

// MN-major (transposed) operand panel, 128-byte swizzle: atoms of 8 K-rows x
// 64 MN elements (1 KB), the K atoms of one 64-wide MN half consecutive, the
// second MN half 8 KB further.
#ifndef FTSP2_MN_LBO
#define FTSP2_MN_LBO 8192
#endif
constexpr uint32_t kMnLbo = FTSP2_MN_LBO;
constexpr uint32_t kMnSbo = FTSP2_MN_LBO == 8192 ? 1024 : 8192;
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kMnLbo >> 4) << 16;     // leading byte offset
    d |= (uint64_t)(kMnSbo >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared variable in CTA `rank`
__device__ __forceinline__ uint32_t map_to(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Arrivals on a barrier of either CTA of the pair.  The barriers only order
// asynchronous-proxy work (TMA completion, tcgen05 commits, TMEM reads fenced
// with tcgen05.fence), so CTA-scope semantics suffice and no cluster-wide
// memory fence is issued per arrival.
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void remote_expect_tx(uint32_t cluster_addr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cluster.b64 _, [%0], %1;" ::"r"(cluster_addr), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
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
// Has the call failed (a wait ran out in this or another CTA)?
__device__ __forceinline__ bool call_failed(const LayerArgs& a) {
    return *reinterpret_cast<volatile int*>(a.status) != 0;
}
__device__ __forceinline__ void record_timeout(const LayerArgs& a) { atomicCAS(a.status, 0, (int)FTSP2_E_TIMEOUT); }

// Wait on a pipeline mbarrier phase.  A failure elsewhere never ends such a
// wait: after a failure every role keeps the barrier protocol of its work list
// (arrivals and commits in the usual order, without loads, MMAs or stores), so
// every phase still completes.  The wait gives up only on its own clock: after
// a.wait_ns it records FTSP2_E_TIMEOUT (the call has failed), and after twice
// that it returns false, which only a broken protocol can cause; the caller
// then leaves its loop and the kernel drains before it frees TMEM.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, const LayerArgs& a) {
    if (try_wait_cluster(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    bool recorded = false;
    for (uint32_t it = 1;; ++it) {
        if (try_wait_cluster(bar, parity)) return true;
        if ((it & 63u) == 0) {
            const unsigned long long dt = globaltimer() - t0;
            if (!recorded && dt > a.wait_ns) {
                record_timeout(a);
                recorded = true;
            }
            if (dt > 2 * a.wait_ns) return false;
        }
    }
}

// TMA 2-D tile load into this CTA's shared memory, completing on an mbarrier
// that may live in the peer CTA of the pair.
__device__ __forceinline__ void tma_load_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                              int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}

template <bool TF32>
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
    }
}

// arrive (once) on the barrier at this shared offset in both CTAs of the pair
// when all previously issued MMAs of this thread have completed
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
    const uint16_t mask = 0x3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}

// arrive on this CTA's barrier only, when all previously issued MMAs of this
// thread (on both CTAs of the pair) have completed
__device__ __forceinline__ void umma_commit_local_pair(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x 16 columns of FP32 from TMEM into registers (no wait)
// single-CTA counterparts
__device__ __forceinline__ void tma_load_one(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
template <bool TF32>
__device__ __forceinline__ void umma_one(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
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
__device__ __forceinline__ void umma_commit_one(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void local_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void local_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* x) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(x[0])), "r"(__float_as_uint(x[1])), "r"(__float_as_uint(x[2])),
                 "r"(__float_as_uint(x[3])), "r"(__float_as_uint(x[4])), "r"(__float_as_uint(x[5])),
                 "r"(__float_as_uint(x[6])), "r"(__float_as_uint(x[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ----------------------------------------------------------------------------------
// Split formats of the next layer's operands (planes of 2- or 4-byte
// elements); the stores themselves are in epi_dgroup_next.
// ----------------------------------------------------------------------------------
template <int FMT>
struct OpFmtT;
template <>
struct OpFmtT<OP_F16X2> {
    static constexpr int NPL = 2, ESZ = 2;
    __device__ static void split(float z, uint32_t* o) {
        const __half h = __float2half_rn(z);
        const __half l = __float2half_rn(z - __half2float(h));
        o[0] = __half_as_ushort(h);
        o[1] = __half_as_ushort(l);
    }
};
template <>
struct OpFmtT<OP_BF16X3> {
    static constexpr int NPL = 3, ESZ = 2;
    __device__ static void split(float z, uint32_t* o) {
        const __nv_bfloat16 b0 = __float2bfloat16_rn(z);
        const float r1 = z - __bfloat162float(b0);
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
        o[0] = __bfloat16_as_ushort(b0);
        o[1] = __bfloat16_as_ushort(b1);
        o[2] = __bfloat16_as_ushort(b2);
    }
};
template <>
struct OpFmtT<OP_TF32X3> {
    static constexpr int NPL = 2, ESZ = 4;
    __device__ static void split(float z, uint32_t* o) {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(z));
        o[0] = hb;
        // the tensor core reads only the TF32 bits of the low part: round it
        // to TF32 (unbiased) instead of letting the low 13 bits be cut
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(o[1]) : "f"(z - __uint_as_float(hb)));
    }
};
template <>
struct OpFmtT<OP_F32> {
    static constexpr int NPL = 1, ESZ = 4;
    __device__ static void split(float z, uint32_t* o) { o[0] = __float_as_uint(z); }
};

template <int ESZ>
__device__ __forceinline__ void store1(uint8_t* dst, uint32_t v) {
    if constexpr (ESZ == 2) *reinterpret_cast<uint16_t*>(dst) = (uint16_t)v;
    else *reinterpret_cast<uint32_t*>(dst) = v;
}
constexpr int kLastLayer = -1;

// What the final epilogue of a non-last layer needs beyond the kernel
// parameters, with the instance's slab offset folded into the pointers (kept
// small).  The accumulator A of a chain sits plane_elems floats after its Z
// (the workspace places them back to back).
struct EpiLite {
    float* Z;          // state slab of Z (blocked layout); A = Z + plane_elems
    uint8_t* op;       // next layer's operand plane 0, slab start (bytes)
    float mul, bp, d, os;
    float p, q, d2;    // next state Z' = p xh + q A, A' = A + d Z + d2 xh (DevLayer)
};

// FMT: operand format written; scaled_in: the products were formed from
// power-of-two scaled FP16 operands (FP16X2 layers).
template <int FMT>
__device__ __forceinline__ void make_lite(const LayerArgs& a, const Tile& t, int g, int k, bool scaled_in, EpiLite& e) {
    const ftsp2_rescale_rec& rec = a.rec[t.inst];
    const DevModel& M = a.models[rec.model];
    const DevLayer L = a.layers[(a.chain_kind[t.chain] == CHAIN_ENTROPY ? M.offS : M.off) + k];
    const size_t slab = (size_t)t.inst * a.P * a.P;
    e.Z = a.Z[t.chain] + slab;
    e.op = (((g - a.gl) & 1) ? a.opw_alt : a.opw)[t.chain] + slab * OpFmtT<FMT>::ESZ;
    e.mul = scaled_in ? L.acc_mul : L.a;
    e.bp = L.bp;
    e.d = L.d;
    e.os = FMT == OP_F16X2 ? L.out_scale : 1.f;
    e.p = L.p;
    e.q = L.q;
    e.d2 = L.d2;
}

// Load the 8 state values of row r, columns c0 .. c0 + 7 (two float4 runs 128
// floats apart in the blocked layout).
__device__ __forceinline__ void load_state8(const float* S, float* x) {
    const float4 u = reinterpret_cast<const float4*>(S)[0], w = reinterpret_cast<const float4*>(S + 128)[0];
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
}
__device__ __forceinline__ void store_state8(float* S, const float* x) {
    reinterpret_cast<float4*>(S)[0] = make_float4(x[0], x[1], x[2], x[3]);
    reinterpret_cast<float4*>(S + 128)[0] = make_float4(x[4], x[5], x[6], x[7]);
}

// 256-bit store (sm_100+): dst must be 32-byte aligned.
__device__ __forceinline__ void st_global_v8(void* dst, const uint32_t* w) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// Where the final epilogue reads a group's sums S and state Z_k, A_k: the
// sums from TMEM and the state from global memory (inline epilogue of the
// accumulating warps), or all three from a shared-memory staging entry in
// the blocked [half][lane][4] layout of the state (deferred epilogue).
struct SrcTmem {
    uint32_t tcol;
    __device__ __forceinline__ void sums(int hh, float* v) const {
        tmem_ld8(tcol + 8 * hh, reinterpret_cast<uint32_t*>(v));
        tmem_wait_ld();
    }
    __device__ __forceinline__ void state(int, const float* Zg, const float* Ag, float* z, float* x) const {
        load_state8(Zg, z);
        load_state8(Ag, x);
    }
};
struct SrcSmem {
    const float* s;    // entry + lane * 4: sums, then Z_k, then A_k (512 floats each)
    __device__ __forceinline__ void sums(int hh, float* v) const { load_state8(s + 256 * hh, v); }
    __device__ __forceinline__ void state(int hh, const float*, const float*, float* z, float* x) const {
        load_state8(s + 512 + 256 * hh, z);
        load_state8(s + 1024 + 256 * hh, x);
    }
};

// Final epilogue of a non-last layer on 16 columns c0 .. c0 + 15 (c0 % 16 == 0)
// of row r, the sums and the state read through src (8-column halves that do
// not touch the triangle or the order are skipped):
//   A_{k+1} = A_k + d_k Z_k,  Z_{k+1} = a_k S + (b_k + 2 a_k tau_k) Z_k,
// then the operands of Z_{k+1} (times the FP16 scale 2^e_{k+1}) for the next
// layer: direct (r, c), r <= c, as one 32-byte vector per plane and lane (full
// sectors; 4-byte formats store two), and mirror (c, r), r < c, one element per
// lane, so that for each column the warp's 32 stores are one contiguous run of
// row c.
template <int FMT, class Src>
__device__ __forceinline__ void epi_dgroup_next(const LayerArgs& a, const EpiLite& e, int n, int R0, int r, int c0,
                                                const Src& src, bool mirror) {
    using F = OpFmtT<FMT>;
    constexpr int ESZ = F::ESZ;
    constexpr int NPL = F::NPL;
    constexpr int WPH = 8 * ESZ / 4;                 // 32-bit words per plane per 8-column half
    const int P = a.P;
    uint32_t wd[NPL][2 * WPH];                       // packed operand words of both halves
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int cg = c0 + 8 * hh;
        if (!(cg < n && cg + kGrp - 1 >= R0)) continue;          // warp-uniform
        float v[8];
        src.sums(hh, v);
        if (r >= n) continue;
        const size_t so = state_off(P, r, cg);
        float* const Zg = e.Z + so;
        float* const Ag = Zg + a.plane_elems;
        float z[8], zn[8];
        src.state(hh, Zg, Ag, z, zn);
        // xh in v, A' in z, Z' in zn (A read before it is replaced)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float xh = fmaf(e.mul, v[u], e.bp * z[u]);
            const float an = fmaf(e.d2, xh, fmaf(e.d, z[u], zn[u]));
            zn[u] = fmaf(e.p, xh, e.q * zn[u]);
            z[u] = an;
        }
        store_state8(Ag, z);
        store_state8(Zg, zn);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t o[NPL];
            F::split(zn[u] * e.os, o);
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
                if constexpr (ESZ == 2) {
                    if (u & 1) wd[p][hh * WPH + u / 2] |= o[p] << 16;
                    else wd[p][hh * WPH + u / 2] = o[p];
                } else {
                    wd[p][hh * WPH + u] = o[p];
                }
                // mirror (c, r), r < c: one contiguous run of row c per column
                const int c = cg + u;
                if (mirror && r < c && c < n)
                    store1<ESZ>(e.op + (size_t)p * a.plane_elems * ESZ + ((size_t)c * P + r) * ESZ, o[p]);
            }
        }
    }
    if (r >= n) return;
    const bool full = r <= c0 && c0 + 15 < n;
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
        uint8_t* const dst = e.op + (size_t)p * a.plane_elems * ESZ + ((size_t)r * P + c0) * ESZ;
        if (full) {
            if constexpr (ESZ == 2) {
                st_global_v8(dst, wd[p]);
            } else {
                st_global_v8(dst, wd[p]);
                st_global_v8(dst + 32, wd[p] + 8);
            }
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = c0 + u;
                if (c < n && r <= c) {
                    const uint32_t val = ESZ == 2 ? ((wd[p][u / 2] >> (16 * (u & 1))) & 0xffffu) : wd[p][u];
                    store1<ESZ>(dst + u * ESZ, val);
                }
            }
        }
    }
}

// Last layer: G = A + d Z + g xh with xh = mul v + bp Z (Eq. mlsp2: A_L + Z_L,
// A_L = A_{L-1} + d Z_{L-1}, Z_L = a v + b' Z_{L-1}; Skip-SP2: A_L + gamma_L x_L)
// (v overwritten with G); rows r >= n give 0.
__device__ __forceinline__ void epi_update_last(const LayerArgs& a, const EpiCtx& e, int r, int c0, float* v) {
    if (r >= e.n) {
#pragma unroll
        for (int u = 0; u < kGrp; ++u) v[u] = 0.f;
        return;
    }
    const size_t so = e.slab + state_off(e.P, r, c0);
    float z[8], x[8];
    load_state8(a.Z[e.chain] + so, z);
    load_state8(a.A[e.chain] + so, x);
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = fmaf(e.L.g, fmaf(e.mul, v[u], e.L.bp * z[u]), fmaf(e.L.d, z[u], x[u]));
}

// Last layer: D = G + f0 I (or (1 - f0) I - G when flipped) at (r, c) and
// (c, r), and the sums of the diagonal and of the squares of G.  The diagonal
// element is added in FP64.  A group's 8 squares are summed without rounding
// error in pairs of FP32 numbers (the product's error by an FMA, each
// addition's by TwoSum, Knuth), the high part is added in FP64 and the low part
// in FP32 into `lo`, which the caller adds once per tile: per-element FP64
// arithmetic would run on the FP64 pipe, the slowest unit of this GPU.  The
// direct row (r, c .. c + 7) is written as two 16-byte vectors when the whole
// group lies in the triangle and is aligned; the mirror (c, r) is one element
// per lane, a contiguous run of row c across the warp.
__device__ __forceinline__ void epi_last(const LayerArgs& a, const EpiCtx& e, int r, int c0, const float* v,
                                         double& tr, double& sq, float& lo) {
    if (r >= e.n) return;
    const bool dout = e.kind == CHAIN_FERMI && a.D;
    float dv[kGrp];
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int jj = 0; jj < kGrp; ++jj) {
        const int c = c0 + jj;
        const float g = v[jj];
        const bool diag = r == c;
        if (e.flip) dv[jj] = (diag ? (float)e.cdiag : 0.f) - g;
        else dv[jj] = g + (diag ? (float)e.cdiag : 0.f);
        if (c < e.n && r <= c) {
            if (diag) tr += (double)g;
            const float w = diag ? g : 2.f * g;            // (r, c) and (c, r)
            const float p = __fmul_rn(w, g);
            const float pe = fmaf(w, g, -p);               // w g - p, exact
            const float t = __fadd_rn(sh, p);
            const float bp = __fsub_rn(t, sh);
            const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));   // sh + p - t, exact
            sh = t;
            sl = __fadd_rn(sl, __fadd_rn(te, pe));
        }
    }
    sq += (double)sh;
    lo = __fadd_rn(lo, sl);
    if (!dout) return;
    float* drow = a.D + e.doff + (int64_t)r * e.n;
    if (c0 >= r && c0 + kGrp <= e.n && (reinterpret_cast<uintptr_t>(drow + c0) & 15u) == 0) {
        reinterpret_cast<float4*>(drow + c0)[0] = make_float4(dv[0], dv[1], dv[2], dv[3]);
        reinterpret_cast<float4*>(drow + c0)[1] = make_float4(dv[4], dv[5], dv[6], dv[7]);
    } else {
#pragma unroll
        for (int jj = 0; jj < kGrp; ++jj) {
            const int c = c0 + jj;
            if (c < e.n && r <= c) drow[c] = dv[jj];
        }
    }
#pragma unroll
    for (int jj = 0; jj < kGrp; ++jj) {
        const int c = c0 + jj;
        if (c < e.n && r < c) a.D[e.doff + (int64_t)c * e.n + r] = dv[jj];
    }
}

// L2 prefetch of the Z and A state that the CTA's epilogue warps read at the
// end of tile tl: rows I*TILE + row0 .. + 127, columns from the diagonal (or the
// tile's first column) to the order n; each 32-row block row of the blocked
// layout is one contiguous run.  Issued by the TMA producer a few K-slices
// before the tile ends.
template <int TILE>
__device__ __forceinline__ void prefetch_tile_state(const LayerArgs& a, const Tile& tl, int row0, int n) {
    const size_t slab = (size_t)tl.inst * a.P * a.P;
    const int cend = min(n, tl.J * TILE + TILE);
#pragma unroll 1
    for (int rb = 0; rb < kCtaRows; rb += 32) {
        const int R = tl.I * TILE + row0 + rb;
        if (R >= n) break;
        const int cs = max(tl.J * TILE, R) & ~7;
        if (cs >= cend) continue;
        const uint32_t bytes = (uint32_t)((cend - cs + 7) / 8) * 1024u;
        const size_t off = slab + state_off(a.P, R, cs);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.Z[tl.chain] + off), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.Z[tl.chain] + a.plane_elems + off), "r"(bytes)
                     : "memory");
    }
}

// ----------------------------------------------------------------------------------
// OUTFMT: operand format written for the next layer, or kLastLayer.
// 16-byte asynchronous global -> shared copies through the load/store path
// (cp.async, L2 only): the store warps' loads do not queue behind the operand
// tiles in the TMA unit.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The persistent loop of a unit visits tiles t, t + nunits, ...: is there an
// active tile after t?  (The last tile of a unit runs its final epilogue inline,
// so that no store-warp tail follows the last MMAs.)
// Work items of a launch: item f is (global layer gl + f / ntiles, tile
// f % ntiles); a one-layer launch has ntiles items.
__device__ __forceinline__ int n_items(const LayerArgs& a) { return a.ntiles * a.nlayers; }
__device__ __forceinline__ void item_of(const LayerArgs& a, int f, int& g, int& t) {
    const int l = f / a.ntiles;
    g = a.gl + l;
    t = f - l * a.ntiles;
}

// Does the unit have an active item after item f?
__device__ __forceinline__ bool has_next_tile(const LayerArgs& a, int f, int nunits) {
    const int nf = n_items(a);
    for (int u = f + nunits; u < nf; u += nunits) {
        int g, t, k;
        item_of(a, u, g, t);
        if (tile_active_g(a, a.tiles[t], g, k)) return true;
    }
    return false;
}

// Completion counters of multi-layer launches, one per (layer, instance,
// chain): an epilogue warp adds its share after its stores (release: fence,
// then the atomic); a reader acquires.  (A counter shared by a whole layer
// took 16 atomics per tile from every CTA on one address, which serialised
// ragged batches of ten thousand tiles per layer.)
__device__ __forceinline__ int* inst_counter(const LayerArgs& a, int g, int inst, int chain) {
    return a.done_inst + ((size_t)g * a.nb + inst) * kMaxChains + chain;
}
__device__ __forceinline__ void done_add(const LayerArgs& a, int g, int inst, int chain, int v) {
    __threadfence();
    atomicAdd(inst_counter(a, g, inst, chain), v);
}
__device__ __forceinline__ int acquire_load(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Wait until the counter at p reaches target.  False when the call has failed
// (this wait ran out after a.wait_ns, which records FTSP2_E_TIMEOUT, or another
// wait of this launch did): the producer then runs its remaining items in skip
// mode, without loads.
__device__ __forceinline__ bool wait_counter(const LayerArgs& a, const int* p, int target) {
    if (acquire_load(p) >= target) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        __nanosleep(256);
        if (acquire_load(p) >= target) return true;
        if (call_failed(a)) return false;
        if (globaltimer() - t0 > a.wait_ns) {
            record_timeout(a);
            return false;
        }
    }
}

// Work items of the deferred epilogue: item i (the block of accumulating warp
// 2 + i) of a tile is 32 rows x EPI_COLS columns; its entries are the 16-column
// groups that touch the triangle and the order.  A cursor (i, g) steps through
// the items i = sw, sw + kStoreWarps, ... of store warp sw.
struct ItemGeo {
    int R0, C0, g_lo, g_hi;
};
template <int TILE, int EPI_COLS>
__device__ __forceinline__ bool item_geo(const Tile& tl, int rank, int n, int i, ItemGeo& ig) {
    const int q = (i + 2) & 3, cq = i >> 2;
    ig.R0 = tl.I * TILE + rank * kCtaRows + q * 32;
    ig.C0 = tl.J * TILE + cq * EPI_COLS;
    if (!(ig.C0 < n && ig.C0 + EPI_COLS - 1 >= ig.R0 && ig.R0 < n)) return false;
    ig.g_lo = ig.R0 > ig.C0 ? min(EPI_COLS / kGrp, (ig.R0 - ig.C0) / kGrp) : 0;
    ig.g_hi = min(EPI_COLS / kGrp, (n - ig.C0 + kGrp - 1) / kGrp);
    return true;
}
template <int TILE, int EPI_COLS>
__device__ __forceinline__ bool next_entry(const Tile& tl, int rank, int n, int& i, int& g) {
    while (i < kEpiWarps) {
        ItemGeo ig;
        if (item_geo<TILE, EPI_COLS>(tl, rank, n, i, ig)) {
            const int gn = g < 0 ? (ig.g_lo & ~1) : g + 2;
            if (gn < ig.g_hi) {
                g = gn;
                return true;
            }
        }
        i += kStoreWarps;
        g = -1;
    }
    return false;
}

template <int MODE, int OUTFMT, bool PAIR, bool DEFER>
__global__ void __launch_bounds__(threads_of(DEFER), 1)
    layer_tc_kernel(const __grid_constant__ LayerArgs a, const __grid_constant__ TmaMaps maps0,
                    const __grid_constant__ TmaMaps maps1) {
    using C = TcCfg<MODE>;
    using G = Geo<PAIR>;
    static_assert(!(DEFER && OUTFMT == kLastLayer), "the last layer runs its epilogue inline");
    constexpr int TILE = G::TILE;
    constexpr int EPI_COLS = TILE / (kEpiWarps / 4);   // columns per epilogue warp (64 or 32)
    constexpr int BKE = 128 / C::ESIZE;                // K elements per 128-byte slice
    constexpr int PLANE = kCtaRows * 128;              // bytes of one 128-row slice
    constexpr int STAGE_BYTES = C::NSPLIT * 2 * PLANE; // A and B planes (B: this CTA's half when PAIR)
    constexpr int KSTEPS = 4;                          // 128-byte slice / 32 bytes per MMA
    constexpr uint32_t IDESC = make_idesc(C::ATYPE, TILE, TILE);
    constexpr int NBUF = G::NBUF;
    constexpr uint32_t TMEM_COLS = NBUF * TILE;

    // A launch whose layers all lie below the first layer any instance starts
    // at (models with fewer layers than the set's maximum start late) has no
    // active item: every thread of both CTAs of a pair leaves at once.
    const int first_layer = *reinterpret_cast<volatile const int*>(a.status + 1);
    if (a.gl + a.nlayers <= first_layer) return;
    // the items of layers before the first active one are skipped by every role
    const int f0 = max(0, first_layer - a.gl) * a.ntiles;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[C::STAGES];
    __shared__ __align__(8) uint64_t empty_bar[C::STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[NBUF];
    __shared__ __align__(8) uint64_t tempty_bar[NBUF];
    // deferred epilogue: scratch full / empty
    __shared__ __align__(8) uint64_t sfull_bar, sempty_bar;
    // drain: the MMA issuer's last commit (all of its MMAs complete)
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_slot;
    // skip mode: set once this CTA has seen the call fail; the roles then keep
    // the barrier protocol of their work items without loads, MMAs or stores
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    // K slices per accumulation chunk at global layer g: the default 128
    // elements, or a shorter chunk requested for the layer
    auto ck_of = [&](int g) {
        const int ce = g >= a.tail_from ? a.chunk_tail : a.chunk_elems;
        return max(1, (ce > 0 ? ce : C::CK * BKE) / BKE);
    };
    const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;     // pair or CTA
    const int nunits = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full_bar[s], G::NCTA);      // one expect_tx arrival per CTA
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < NBUF; ++s) {
            mbar_init(&tfull_bar[s], 1);
            mbar_init(&tempty_bar[s], G::NCTA * kEpiWarps);
        }
        if constexpr (DEFER) {
            mbar_init(&sfull_bar, kEpiWarps);
            mbar_init(&sempty_bar, kStoreWarps);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            // (layer, instance) of each chain whose predecessor is known complete
            int known_g[kMaxChains] = {-1, -1}, known_i[kMaxChains] = {-1, -1};
            bool skip = false;                       // the call has failed: no more loads
            bool broken = false;                     // a pipeline wait ran out twice
            const int nf = n_items(a);
            for (int f = f0 + unit; f < nf && !broken; f += nunits) {
                int g, t;
                item_of(a, f, g, t);
                const Tile tl = a.tiles[t];
                int k;
                if (!tile_active_g(a, tl, g, k)) {
                    // an inactive item counts as finished for the layer's completion
                    if (a.nlayers > 1) atomicAdd(inst_counter(a, g, tl.inst, tl.chain), kEpiWarps);
                    continue;
                }
                // only multi-layer launches wait on other CTAs and can fail
                if (!skip && a.nlayers > 1 && call_failed(a)) skip = true;
                if (!skip && g > a.gl && g - 1 >= first_layer &&
                    !(g == known_g[tl.chain] && tl.inst == known_i[tl.chain])) {
                    // Operands and state of this item were written by other CTAs:
                    // wait for the previous layer of its own instance only, so a
                    // small instance need not wait for a large one.
                    const int tgt = kEpiWarps * G::NCTA * a.iw[tl.inst].tile_count[a.dtab][tl.chain] +
                                    (g == a.stall_layer ? 1 : 0);
                    if (wait_counter(a, inst_counter(a, g - 1, tl.inst, tl.chain), tgt)) {
                        known_g[tl.chain] = g;
                        known_i[tl.chain] = tl.inst;
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    } else {
                        skip = true;
                    }
                }
                if (skip) *reinterpret_cast<volatile int*>(&abort_flag) = 1;
                const TmaMaps& maps = ((g - a.gl) & 1) ? maps1 : maps0;
                const int n = a.inst[tl.inst].n;
                const int nk = (n + BKE - 1) / BKE;
                const int rowA = tl.inst * a.P + tl.I * TILE + (int)rank * kCtaRows;
                const int rowB = tl.inst * a.P + tl.J * TILE + (int)rank * kCtaRows;
                // transposed panels: MN index (column of the stored upper block)
                const int mnA = tl.I * TILE + (int)rank * kCtaRows, mnB = tl.J * TILE + (int)rank * kCtaRows;
                for (int kb = 0; kb < nk; ++kb) {
                    // K-slices left of a panel's diagonal block: not stored below
                    // the diagonal, loaded from the transposed upper block
                    const bool lowA = !C::TF32 && a.lower_t && kb * BKE + BKE <= tl.I * TILE;
                    const bool lowB = !C::TF32 && a.lower_t && kb * BKE + BKE <= tl.J * TILE;
                    const int krow = tl.inst * a.P + kb * BKE;
                    if (!wait_bar(&empty_bar[stage], phase ^ 1u, a)) {
                        broken = true;
                        break;
                    }
                    uint8_t* sbase = smem + stage * STAGE_BYTES;
                    if constexpr (PAIR) {
                        const uint32_t fb = map_to(smem_u32(&full_bar[stage]), 0);
                        if (skip) {
                            // the stage's arrival without data: the phase completes
                            // with the peer's loads (if any) and no MMA reads it
                            remote_arrive(fb);
                        } else {
                            if (kb == max(0, nk - 3)) prefetch_tile_state<TILE>(a, tl, (int)rank * kCtaRows, n);
                            remote_expect_tx(fb, STAGE_BYTES);
#pragma unroll
                            for (int s = 0; s < C::NSPLIT; ++s) {
                                const uint32_t dA = smem_u32(sbase + s * PLANE), dB = smem_u32(sbase + (C::NSPLIT + s) * PLANE);
                                if (lowA) {
                                    tma_load_pair(dA, &maps.t[tl.chain][s], fb, mnA, krow);
                                    tma_load_pair(dA + PLANE / 2, &maps.t[tl.chain][s], fb, mnA + 64, krow);
                                } else {
                                    tma_load_pair(dA, &maps.a[tl.chain][s], fb, kb * BKE, rowA);
                                }
                                if (lowB) {
                                    tma_load_pair(dB, &maps.t[tl.chain][s], fb, mnB, krow);
                                    tma_load_pair(dB + PLANE / 2, &maps.t[tl.chain][s], fb, mnB + 64, krow);
                                } else {
                                    tma_load_pair(dB, &maps.a[tl.chain][s], fb, kb * BKE, rowB);
                                }
                            }
                        }
                    } else {
                        const uint32_t fb = smem_u32(&full_bar[stage]);
                        if (skip) {
                            local_arrive(fb);
                        } else {
                            if (kb == max(0, nk - 3)) prefetch_tile_state<TILE>(a, tl, (int)rank * kCtaRows, n);
                            local_expect_tx(fb, STAGE_BYTES);
#pragma unroll
                            for (int s = 0; s < C::NSPLIT; ++s) {
                                const uint32_t dA = smem_u32(sbase + s * PLANE), dB = smem_u32(sbase + (C::NSPLIT + s) * PLANE);
                                if (lowA) {
                                    tma_load_one(dA, &maps.t[tl.chain][s], fb, mnA, krow);
                                    tma_load_one(dA + PLANE / 2, &maps.t[tl.chain][s], fb, mnA + 64, krow);
                                } else {
                                    tma_load_one(dA, &maps.a[tl.chain][s], fb, kb * BKE, rowA);
                                }
                                if (lowB) {
                                    tma_load_one(dB, &maps.t[tl.chain][s], fb, mnB, krow);
                                    tma_load_one(dB + PLANE / 2, &maps.t[tl.chain][s], fb, mnB + 64, krow);
                                } else {
                                    tma_load_one(dB, &maps.a[tl.chain][s], fb, kb * BKE, rowB);
                                }
                            }
                        }
                    }
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (broken) {
                // The barrier protocol failed, so the completion of the loads
                // already issued cannot be observed: give them a bounded grace
                // period (a load of one stage takes microseconds) before the
                // CTA releases its shared memory.
                *reinterpret_cast<volatile int*>(&abort_flag) = 1;
                const unsigned long long t0 = globaltimer();
                while (globaltimer() - t0 < 2000000ull) __nanosleep(1000);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer (the even CTA of a pair) ----------------
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            // descriptors differ only in the start-address field (bits 0-13,
            // address >> 4); all operand slices lie inside this CTA's window
            const uint64_t desc0 = sdesc_sw128(smem_u32(smem));
            const uint64_t descT = sdesc_mn_sw128(smem_u32(smem));   // transposed panels
            const int nf = n_items(a);
            for (int f = f0 + unit; f < nf && ok; f += nunits) {
                int g, t;
                item_of(a, f, g, t);
                const Tile tl = a.tiles[t];
                int k;
                if (!tile_active_g(a, tl, g, k)) continue;
                const int n = a.inst[tl.inst].n;
                const int nk = (n + BKE - 1) / BKE;
                const int ck = ck_of(g);
                for (int kc = 0; kc < nk && ok; kc += ck) {
                    if (!wait_bar(&tempty_bar[buf], aphase ^ 1u, a)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)(buf * TILE);
                    const int kend = min(nk, kc + ck);
                    for (int kb = kc; kb < kend; ++kb) {
                        if (!wait_bar(&full_bar[stage], phase, a)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        // skip mode: the stage holds no new data; the commits below
                        // keep the protocol
                        const bool mma = *reinterpret_cast<volatile int*>(&abort_flag) == 0;
                        const uint64_t ds = desc0 + (uint64_t)((stage * STAGE_BYTES) >> 4);
                        const uint64_t dsT = descT + (uint64_t)((stage * STAGE_BYTES) >> 4);
                        const uint32_t first = kb == kc ? 0u : 1u;
                        // the producer's classification of this K-slice (transposed
                        // panels: MN-major operand, K steps of two 1 KB atoms)
                        const bool lowA = !C::TF32 && a.lower_t && kb * BKE + BKE <= tl.I * TILE;
                        const bool lowB = !C::TF32 && a.lower_t && kb * BKE + BKE <= tl.J * TILE;
                        const uint32_t idesc = IDESC | (lowA ? 1u << 15 : 0u) | (lowB ? 1u << 16 : 0u);
                        const uint64_t baseA = lowA ? dsT : ds, baseB = lowB ? dsT : ds;
                        const uint32_t stepA = lowA ? 2048u : 32u, stepB = lowB ? 2048u : 32u;
                        // The small products (index sum >= 1) of the slice go first and
                        // the leading one (p = 0) last: in a chunk's first slice the
                        // small products are added while the accumulator holds only
                        // small values, so fewer additions land on a large partial sum
                        // (the tensor core's FP32 accumulation is not round-to-nearest).
                        // Measured: 15-30 % smaller errors in D and S at the same speed.
#pragma unroll
                        for (int q = 0; q < C::NPROD; ++q) {
                            const int p = C::NPROD - 1 - q;
#pragma unroll
                            for (int kk = 0; kk < KSTEPS && mma; ++kk) {
                                const uint64_t da = baseA + (uint64_t)((prod_a(p) * PLANE + kk * stepA) >> 4);
                                const uint64_t db = baseB + (uint64_t)(((C::NSPLIT + prod_b(p)) * PLANE + kk * stepB) >> 4);
                                if constexpr (PAIR)
                                    umma_pair<C::TF32>(dt, da, db, idesc, (kk == 0 && q == 0) ? first : 1u);
                                else
                                    umma_one<C::TF32>(dt, da, db, idesc, (kk == 0 && q == 0) ? first : 1u);
                            }
                        }
                        if constexpr (PAIR) umma_commit_pair(smem_u32(&empty_bar[stage]));
                        else umma_commit_one(smem_u32(&empty_bar[stage]));
                        if (++stage == C::STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    if constexpr (PAIR) umma_commit_pair(smem_u32(&tfull_bar[buf]));
                    else umma_commit_one(smem_u32(&tfull_bar[buf]));
                    if (++buf == NBUF) {
                        buf = 0;
                        aphase ^= 1u;
                    }
                }
            }
            // Drain: every MMA this thread issued (they write TMEM of both CTAs
            // of a pair and read both CTAs' stages) has completed before the
            // final barrier, after which the CTAs free TMEM and shared memory.
            if constexpr (PAIR) umma_commit_local_pair(smem_u32(&drain_bar));
            else umma_commit_one(smem_u32(&drain_bar));
            if (!wait_bar(&drain_bar, 0, a)) {
                const unsigned long long t0 = globaltimer();
                while (globaltimer() - t0 < 2000000ull) __nanosleep(1000);
            }
        }
        __syncwarp();
    } else if (DEFER && warp >= 2 + kEpiWarps) {
        // ---------------- deferred final epilogue (store warps) ----------------
        // Tile t's finished sums arrive in the CTA's scratch while the MMAs and
        // the accumulating warps already work on tile t + 1.  Each lane streams
        // its rows of the entries (sums, Z_k, A_k of 16 columns) into a
        // two-deep shared ring with cp.async; the warp computes Z_{k+1},
        // A_{k+1} and the next operands one entry at a time.
        if constexpr (DEFER) {
        const int sw = warp - 2 - kEpiWarps;
        uint8_t* const ring = smem + C::STAGES * STAGE_BYTES + sw * (kRing * kEntryBytes);
        const float* const scr = a.escr + (size_t)blockIdx.x * kEpiScratchFloats;
        uint32_t sp = 0;
        uint32_t used = 0;                       // entries consumed (ring slot)
        bool ok = true;
        const int nf = n_items(a);
        for (int f = f0 + unit; f < nf && ok; f += nunits) {
            int g, t;
            item_of(a, f, g, t);
            const Tile tl = a.tiles[t];
            int k;
            if (!tile_active_g(a, tl, g, k)) continue;
            if (!has_next_tile(a, f, nunits)) continue;     // inline in the accumulating warps
            if (!wait_bar(&sfull_bar, sp, a)) {
                ok = false;
                break;
            }
            sp ^= 1u;
            // skip mode (warp-uniform): hand the scratch back without the work
            const bool work = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&abort_flag) == 0 ? 1 : 0, 0) != 0;
            if (work) {
            if (a.nlayers > 1 && g > a.gl) {
                // the state of layer g - 1 of this instance, written by other CTAs
                if (lane == 0) acquire_load(inst_counter(a, g - 1, tl.inst, tl.chain));
                __syncwarp();
            }
            const int n = a.inst[tl.inst].n;
            EpiLite e;
            make_lite<OUTFMT>(a, tl, g, k, MODE == FTSP2_FP16X2, e);
            // each lane copies exactly the 16-byte runs it reads later (its row
            // of the 8-column halves), so its own cp.async.wait_group suffices
            auto issue = [&](int i, int g, uint32_t slot) {
                ItemGeo ig;
                item_geo<TILE, EPI_COLS>(tl, (int)rank, n, i, ig);
                const int c0 = ig.C0 + kGrp * g;
                const bool two = c0 + kGrp < n;          // second 8-column block inside the order
                const uint32_t dst = smem_u32(ring + slot * kEntryBytes) + 16u * lane;
                const float* ssrc = scr + i * kItemFloats + g * 256 + lane * 4;
                const float* zsrc = e.Z + state_off(a.P, ig.R0, c0) + lane * 4;
#pragma unroll
                for (int o = 0; o < 512; o += 128) {
                    cp_async16(dst + 4u * o, ssrc + o);
                    if (o < 256 || two) {
                        cp_async16(dst + 4u * (512 + o), zsrc + o);
                        cp_async16(dst + 4u * (1024 + o), zsrc + a.plane_elems + o);
                    }
                }
                cp_async_commit();
            };
            int ii = sw, gi = -1, iu = sw, gu = -1;
            uint32_t pending = 0;                // copy groups in flight
            bool more = next_entry<TILE, EPI_COLS>(tl, (int)rank, n, ii, gi);
            for (uint32_t s = 0; s < (uint32_t)kRing && more; ++s) {
                issue(ii, gi, (used + s) % kRing);
                ++pending;
                more = next_entry<TILE, EPI_COLS>(tl, (int)rank, n, ii, gi);
            }
            while (next_entry<TILE, EPI_COLS>(tl, (int)rank, n, iu, gu)) {
                const uint32_t slot = used % kRing;
                if (pending > 1) cp_async_wait<1>();
                else cp_async_wait<0>();
                --pending;
                ItemGeo ig;
                item_geo<TILE, EPI_COLS>(tl, (int)rank, n, iu, ig);
                const SrcSmem src{reinterpret_cast<const float*>(ring + slot * kEntryBytes) + lane * 4};
                epi_dgroup_next<OUTFMT>(a, e, n, ig.R0, ig.R0 + lane, ig.C0 + kGrp * gu, src,
                                        a.mirror_all || tl.I == tl.J);
                __syncwarp();                    // every lane is done with the slot
                ++used;
                if (more) {
                    issue(ii, gi, (used + kRing - 1) % kRing);
                    ++pending;
                    more = next_entry<TILE, EPI_COLS>(tl, (int)rank, n, ii, gi);
                }
            }
            }
            __syncwarp();
            if (lane == 0) {
                // this warp's share of the tile's kEpiWarps completions
                if (a.nlayers > 1) done_add(a, g, tl.inst, tl.chain, kEpiWarps / kStoreWarps);
                local_arrive(smem_u32(&sempty_bar));
            }
        }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..17) ----------------
        const int q = warp & 3;                  // TMEM lane quarter
        const int cq = (warp - 2) >> 2;          // column quarter of the tile
        // "tempty" barriers of the even CTA (consecutive 8-byte words)
        const uint32_t tempty0 = PAIR ? map_to(smem_u32(&tempty_bar[0]), 0) : smem_u32(&tempty_bar[0]);
        int buf = 0;
        uint32_t aphase = 0;
        uint32_t sp = 0;                         // scratch parity (deferred epilogue)
        bool ok = true;
        const int nf = n_items(a);
        for (int f = f0 + unit; f < nf && ok; f += nunits) {
            int g, t;
            item_of(a, f, g, t);
            // Only the chunk count and the liveness of the warp's block are
            // carried through the drain loop; the tile's descriptor and the
            // rest of the context are fetched again for the final epilogue
            // (keeps the drain loop of a pair tile, with its 64 accumulator
            // registers, free of spills).
            int nch;
            bool warp_live, defer_tile;
            {
                const Tile tl = a.tiles[t];
                int k;
                if (!tile_active_g(a, tl, g, k)) continue;
                const int n = a.inst[tl.inst].n;
                const int R0 = tl.I * TILE + (int)rank * kCtaRows + q * 32;
                const int C0 = tl.J * TILE + cq * EPI_COLS;
                warp_live = C0 < n && C0 + EPI_COLS - 1 >= R0 && R0 < n;
                const int ck = ck_of(g);
                nch = ((n + BKE - 1) / BKE + ck - 1) / ck;
                defer_tile = DEFER && has_next_tile(a, f, nunits);
            }
            float acc[EPI_COLS];
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) acc[i] = 0.f;
            // Chunk drain.  Chunks 0 .. nch - 2 are added into acc and their
            // buffer released at once.  The last chunk is added too, and the
            // finished sum is written back into that chunk's TMEM buffer, which
            // stays held through the final epilogue: the epilogue then reads
            // its 8-column groups from TMEM, so the 64 accumulator registers of
            // a pair tile are free for the memory work.  The MMAs of the next
            // tile meanwhile fill the other buffers.
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cq * EPI_COLS);
            for (int j = 0; j < nch; ++j) {
                if (!wait_bar(&tfull_bar[buf], aphase, a)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tbase + (uint32_t)(buf * TILE);
                if (warp_live) {
#pragma unroll
                    for (int g = 0; g < EPI_COLS / 16; ++g) {
                        uint32_t v[16];
                        tmem_ld16(ta + 16 * g, v);
                        tmem_wait_ld();
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) acc[16 * g + jj] += __uint_as_float(v[jj]);
                    }
                }
                if (j == nch - 1 && !defer_tile) {
                    if (warp_live) {
#pragma unroll
                        for (int g = 0; g < EPI_COLS / 8; ++g) tmem_st8(ta + 8 * g, &acc[8 * g]);
                        tmem_wait_st();
                    }
                    break;                            // buffer released after the final epilogue
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR) remote_arrive(tempty0 + 8u * (uint32_t)buf);
                    else local_arrive(tempty0 + 8u * (uint32_t)buf);
                }
                if (++buf == NBUF) {
                    buf = 0;
                    aphase ^= 1u;
                }
            }
            if (!ok) break;
            // skip mode (warp-uniform): the protocol without the memory work
            const bool work = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(&abort_flag) == 0 ? 1 : 0, 0) != 0;
            if (defer_tile) {
                // hand the finished sums to the store warps through the scratch
                // (its previous tile must have been read), then go on to the next tile
                if (!wait_bar(&sempty_bar, sp ^ 1u, a)) break;
                sp ^= 1u;
                if (warp_live && work) {
                    float* const dst = a.escr + (size_t)blockIdx.x * kEpiScratchFloats + (warp - 2) * kItemFloats + lane * 4;
#pragma unroll
                    for (int g = 0; g < EPI_COLS / 8; ++g) store_state8(dst + 256 * g, &acc[8 * g]);
                }
                __syncwarp();
                if (lane == 0) local_arrive(smem_u32(&sfull_bar));
                continue;
            }
            const uint32_t tfin = tbase + (uint32_t)(buf * TILE);   // the held buffer
            const Tile tl = a.tiles[t];
            int k;
            tile_active_g(a, tl, g, k);
            if (a.nlayers > 1 && g > a.gl) {
                // the state of layer g - 1 of this instance, written by other CTAs
                if (lane == 0) acquire_load(inst_counter(a, g - 1, tl.inst, tl.chain));
                __syncwarp();
            }
            const int n = a.inst[tl.inst].n;
            const int R0 = tl.I * TILE + (int)rank * kCtaRows + q * 32;   // first row of this warp
            const int r = R0 + lane;
            const int C0 = tl.J * TILE + cq * EPI_COLS;                   // first column of this warp
            double tr = 0.0, sq = 0.0;
            float sq_lo = 0.f;
            if (warp_live && work) {
                if constexpr (OUTFMT == kLastLayer) {
                    EpiCtx e;
                    make_ctx(a, tl, k, e, MODE == FTSP2_FP16X2);
#pragma unroll 1
                    for (int g = 0; g < EPI_COLS / kGrp; ++g) {
                        const int c0 = C0 + kGrp * g;
                        if (c0 < e.n && c0 + kGrp - 1 >= R0) {
                            float v[8];
                            tmem_ld8(tfin + 8 * g, reinterpret_cast<uint32_t*>(v));
                            tmem_wait_ld();
                            epi_update_last(a, e, r, c0, v);
                            epi_last(a, e, r, c0, v, tr, sq, sq_lo);
                        }
                    }
                } else {
                    EpiLite e;
                    make_lite<OUTFMT>(a, tl, g, k, MODE == FTSP2_FP16X2, e);
                    // the groups that touch the triangle and the order form one range
                    const int g_lo = R0 > C0 ? min(EPI_COLS / kGrp, (R0 - C0) / kGrp) : 0;
                    const int g_hi = min(EPI_COLS / kGrp, (n - C0 + kGrp - 1) / kGrp);
#pragma unroll 1
                    for (int g = g_lo & ~1; g < g_hi; g += 2)
                        epi_dgroup_next<OUTFMT>(a, e, n, R0, r, C0 + kGrp * g, SrcTmem{tfin + 8 * g},
                                                a.mirror_all || tl.I == tl.J);
                }
            }
            // release the held accumulator buffer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if constexpr (PAIR) remote_arrive(tempty0 + 8u * (uint32_t)buf);
                else local_arrive(tempty0 + 8u * (uint32_t)buf);
                if (a.nlayers > 1) done_add(a, g, tl.inst, tl.chain, 1);
            }
            if (++buf == NBUF) {
                buf = 0;
                aphase ^= 1u;
            }
            if constexpr (OUTFMT == kLastLayer) {
                sq += (double)sq_lo;
                for (int o = 16; o > 0; o >>= 1) {
                    tr += __shfl_xor_sync(0xffffffffu, tr, o);
                    sq += __shfl_xor_sync(0xffffffffu, sq, o);
                }
                if (lane == 0) {
                    const int slot = (int)rank * kEpiWarps + (warp - 2);
                    a.partials[((size_t)t * kPartialSlots + slot) * 2 + 0] = tr;
                    a.partials[((size_t)t * kPartialSlots + slot) * 2 + 1] = sq;
                    if constexpr (!PAIR) {
                        // a single CTA fills half of the tile's slots; the finalize sums all
                        a.partials[((size_t)t * kPartialSlots + slot + kEpiWarps) * 2 + 0] = 0.0;
                        a.partials[((size_t)t * kPartialSlots + slot + kEpiWarps) * 2 + 1] = 0.0;
                    }
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
    }
}

int tc_block_n(int, int pair) { return pair ? Geo<true>::TILE : Geo<false>::TILE; }
int tc_block_m(int, int pair) { return pair ? Geo<true>::TILE : Geo<false>::TILE; }

template <int MODE>
static int smem_of(bool deferred = false) {
    using C = TcCfg<MODE>;
    return C::STAGES * C::NSPLIT * 2 * kCtaRows * 128 + 1024 + (deferred ? kStoreWarps * kRing * kEntryBytes : 0);
}

int tc_smem_bytes(int mode) {
    switch (mode) {
        case FTSP2_FP16X2: return smem_of<FTSP2_FP16X2>();
        case FTSP2_BF16X3: return smem_of<FTSP2_BF16X3>();
        case FTSP2_TF32X3: return smem_of<FTSP2_TF32X3>();
    }
    return 0;
}

template <int MODE, int OUTFMT, bool PAIR, bool DEFER>
static cudaError_t set_smem_attr() {
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(layer_tc_kernel<MODE, OUTFMT, PAIR, DEFER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_of<MODE>(DEFER));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    return cudaSuccess;
}

// A multi-layer launch (a.nlayers > 1) is cooperative: its CTAs wait on one
// another, so all of them must be resident at once.
template <int MODE, int OUTFMT, bool PAIR, bool DEFER>
static cudaError_t launch_variant(const LayerArgs& a, const TmaMaps& maps, const TmaMaps& maps_alt, int units,
                                  cudaStream_t s) {
    const int smem = smem_of<MODE>(DEFER);
    cudaError_t e = set_smem_attr<MODE, OUTFMT, PAIR, DEFER>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Geo<PAIR>::NCTA * units, 1, 1);
    cfg.blockDim = dim3(threads_of(DEFER), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (PAIR) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = Geo<PAIR>::NCTA;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (a.nlayers > 1) {
        attr[na].id = cudaLaunchAttributeCooperative;
        attr[na].val.cooperative = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    e = cudaLaunchKernelEx(&cfg, layer_tc_kernel<MODE, OUTFMT, PAIR, DEFER>, a, maps, maps_alt);
    count_launch();
    return e;
}

template <int MODE, int OUTFMT, bool PAIR, bool DEFER>
static int max_units_variant() {
    if (set_smem_attr<MODE, OUTFMT, PAIR, DEFER>() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Geo<PAIR>::NCTA, 1, 1);
    cfg.blockDim = dim3(threads_of(DEFER), 1, 1);
    cfg.dynamicSmemBytes = smem_of<MODE>(DEFER);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Geo<PAIR>::NCTA;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, layer_tc_kernel<MODE, OUTFMT, PAIR, DEFER>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int MODE, int MAINFMT, bool PAIR>
static cudaError_t launch_shape(const LayerArgs& a, const TmaMaps& maps, const TmaMaps& maps_alt, int units,
                                cudaStream_t s) {
    if (a.last) return launch_variant<MODE, kLastLayer, PAIR, false>(a, maps, maps_alt, units, s);
    if (a.next_fmt == OP_F32) return launch_variant<MODE, OP_F32, PAIR, false>(a, maps, maps_alt, units, s);
    if constexpr (MAINFMT != OP_BF16X3) {
        // the layer before BF16X3 refinement layers (FTSP2_REFINE_TC)
        if (a.next_fmt == OP_BF16X3) return launch_variant<MODE, OP_BF16X3, PAIR, false>(a, maps, maps_alt, units, s);
    }
    // the layers of the main format: the final epilogue inline or deferred to
    // store warps (a.escr set: a scratch slot for each CTA of the grid)
    if constexpr (PAIR) {
        if (a.escr) return launch_variant<MODE, MAINFMT, PAIR, true>(a, maps, maps_alt, units, s);
    }
    return launch_variant<MODE, MAINFMT, PAIR, false>(a, maps, maps_alt, units, s);
}

template <int MODE, int MAINFMT>
static cudaError_t launch_mode(const LayerArgs& a, const TmaMaps& maps, const TmaMaps& maps_alt, int units, int pair,
                               cudaStream_t s) {
    return pair ? launch_shape<MODE, MAINFMT, true>(a, maps, maps_alt, units, s)
                : launch_shape<MODE, MAINFMT, false>(a, maps, maps_alt, units, s);
}

cudaError_t launch_layer_tc(int mode, const LayerArgs& a, const TmaMaps& maps, const TmaMaps& maps_alt, int units,
                            int pair, cudaStream_t s) {
    switch (mode) {
        case FTSP2_FP16X2: return launch_mode<FTSP2_FP16X2, OP_F16X2>(a, maps, maps_alt, units, pair, s);
        case FTSP2_BF16X3: return launch_mode<FTSP2_BF16X3, OP_BF16X3>(a, maps, maps_alt, units, pair, s);
        case FTSP2_TF32X3: return launch_mode<FTSP2_TF32X3, OP_TF32X3>(a, maps, maps_alt, units, pair, s);
    }
    return cudaErrorInvalidValue;
}

template <int MODE, int MAINFMT>
static int max_units_mode(int pair, bool defer) {
    if (pair) {
        return defer ? max_units_variant<MODE, MAINFMT, true, true>() : max_units_variant<MODE, MAINFMT, true, false>();
    }
    return max_units_variant<MODE, MAINFMT, false, false>();
}

int layer_tc_max_units(int mode, int pair, bool defer) {
    switch (mode) {
        case FTSP2_FP16X2: return max_units_mode<FTSP2_FP16X2, OP_F16X2>(pair, defer);
        case FTSP2_BF16X3: return max_units_mode<FTSP2_BF16X3, OP_BF16X3>(pair, defer);
        case FTSP2_TF32X3: return max_units_mode<FTSP2_TF32X3, OP_TF32X3>(pair, defer);
    }
    return 0;
}

}  // namespace ftsp2
