// (a3)-(a6) One layer of the centred recursion with FP32 FMA products on the
// CUDA cores: the FTSP2_FP32 mode and the FP32 refinement layers
// (FTSP2_REFINE1/2).  Same triangular tile list (128 x 128 tiles), same
// epilogue as the tensor-core kernel (plus the Max-SP2 layers, which only this
// kernel runs); the operand is the full symmetric FP32 matrix Z_k (written for
// this layer by the previous layer's epilogue).
// Classic register-blocked tile product: 256 threads, 8 x 8 outputs each,
// K-slices of 16 staged through shared memory (transposed, K-major rows),
// sums taken over 128-element K chunks.
#include "epilogue.cuh"
#include "ftsp2_internal.h"

namespace ftsp2 {

constexpr int SB = 128;   // tile edge
constexpr int SK = 16;    // K slice

__global__ void __launch_bounds__(256) layer_simt_kernel(const __grid_constant__ LayerArgs a) {
    __shared__ __align__(16) float As[SK][SB + 4];
    __shared__ __align__(16) float Bs[SK][SB + 4];
    __shared__ double red[8][2];
    // no instance starts before status[1]: a layer below it has nothing to do
    if (a.gl < *reinterpret_cast<volatile const int*>(a.status + 1)) return;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const Tile tl = a.tiles[t];
        int k;
        if (!tile_active(a, tl, k)) continue;
        const int n = a.inst[tl.inst].n;
        const float* Op = reinterpret_cast<const float*>(a.opr[tl.chain]) + (size_t)tl.inst * a.P * a.P;
        const int rowA = tl.I * SB, rowB = tl.J * SB;
        // products are summed over 128-element K chunks in `part` and the
        // chunks are added into `acc` (shorter FP32 accumulation runs)
        float acc[8][8], part[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = part[i][j] = 0.f;
        const int nk = (n + SK - 1) / SK;
        // loader mapping: 128 rows x 16 columns = 512 float4; 2 per thread
        for (int kb = 0; kb < nk; ++kb) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int idx = tid + h * 256;      // 0..511
                const int row = idx >> 2, c4 = (idx & 3) * 4;
                const float4 va = *reinterpret_cast<const float4*>(Op + (size_t)(rowA + row) * a.P + kb * SK + c4);
                const float4 vb = *reinterpret_cast<const float4*>(Op + (size_t)(rowB + row) * a.P + kb * SK + c4);
                As[c4 + 0][row] = va.x; As[c4 + 1][row] = va.y; As[c4 + 2][row] = va.z; As[c4 + 3][row] = va.w;
                Bs[c4 + 0][row] = vb.x; Bs[c4 + 1][row] = vb.y; Bs[c4 + 2][row] = vb.z; Bs[c4 + 3][row] = vb.w;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < SK; ++kk) {
                float ra[8], rb[8];
                const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
                ra[0] = a0.x; ra[1] = a0.y; ra[2] = a0.z; ra[3] = a0.w;
                ra[4] = a1.x; ra[5] = a1.y; ra[6] = a1.z; ra[7] = a1.w;
                rb[0] = b0.x; rb[1] = b0.y; rb[2] = b0.z; rb[3] = b0.w;
                rb[4] = b1.x; rb[5] = b1.y; rb[6] = b1.z; rb[7] = b1.w;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) part[i][j] = fmaf(ra[i], rb[j], part[i][j]);
            }
            __syncthreads();
            if ((kb & 7) == 7 || kb == nk - 1) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        acc[i][j] += part[i][j];
                        part[i][j] = 0.f;
                    }
            }
        }
        EpiCtx e;
        make_ctx(a, tl, k, e, false);
        double tr = 0.0, sq = 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = rowA + ty * 8 + i;
            const int c0 = rowB + tx * 8;
            if (c0 < n && c0 + 7 >= r) {
                if (e.L.nplanes > 0) epi_segment_max<8>(a, e, r, c0, acc[i], tr, sq);
                else epi_segment<8>(a, e, r, c0, acc[i], tr, sq);
            }
        }
        if (a.last) {
            for (int o = 16; o > 0; o >>= 1) {
                tr += __shfl_xor_sync(0xffffffffu, tr, o);
                sq += __shfl_xor_sync(0xffffffffu, sq, o);
            }
            if ((tid & 31) == 0) {
                red[tid >> 5][0] = tr;
                red[tid >> 5][1] = sq;
            }
            __syncthreads();
            if (tid < kPartialSlots) {
                // one slot per warp; the remaining slots of the tile hold zeros
                a.partials[((size_t)t * kPartialSlots + tid) * 2 + 0] = tid < 8 ? red[tid][0] : 0.0;
                a.partials[((size_t)t * kPartialSlots + tid) * 2 + 1] = tid < 8 ? red[tid][1] : 0.0;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_layer_simt(const LayerArgs& a, int grid, cudaStream_t s) {
    layer_simt_kernel<<<grid, 256, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace ftsp2
