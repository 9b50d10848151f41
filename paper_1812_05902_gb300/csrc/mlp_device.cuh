// Device routines of the MLP shared by the training kernels (mlp.cu) and the
// fused surrogate render kernel (surrogate.cu): warp-level BF16 mma.sync
// m16n8k16 with ldmatrix operand loads, and the per-warp forward of a
// 16-row tile with the network resident in shared memory.
#pragma once

#include <cuda_bf16.h>

#include "mlp.cuh"

namespace pivbos {
namespace mlpd {

constexpr int kThreads = 256;   // 8 warps per CTA in the MLP kernels
constexpr int kPadH = kMlpHidden + 8;   // padded row (bank-conflict-free ldmatrix)
constexpr int kPadIn = kMlpIn + 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma16816(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Shared-memory image of the network for the forward kernel.
struct FwdSmem {
    __nv_bfloat16 w0[kMlpHidden * kPadIn];
    __nv_bfloat16 w123[3][kMlpHidden * kPadH];
    __nv_bfloat16 w4[8 * kPadH];
    float bias[kMlpLayers][kMlpHidden];
    __nv_bfloat16 act[8][2][16 * kPadH];   // per warp, ping-pong
};

__device__ inline void load_network(FwdSmem& S, const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params)
{
    // layer 0: [128][16]
    for (int e = threadIdx.x; e < kMlpHidden * kMlpIn; e += blockDim.x) {
        const int o = e / kMlpIn, i = e % kMlpIn;
        S.w0[o * kPadIn + i] = wbf[mlp_wbf_offset(0) + e];
    }
    for (int l = 1; l <= 3; ++l)
        for (int e = threadIdx.x; e < kMlpHidden * kMlpHidden; e += blockDim.x) {
            const int o = e / kMlpHidden, i = e % kMlpHidden;
            S.w123[l - 1][o * kPadH + i] = wbf[mlp_wbf_offset(l) + e];
        }
    // layer 4: [4][128] padded to 8 rows
    for (int e = threadIdx.x; e < 8 * kMlpHidden; e += blockDim.x) {
        const int o = e / kMlpHidden, i = e % kMlpHidden;
        S.w4[o * kPadH + i] = o < kMlpOut ? wbf[mlp_wbf_offset(4) + o * kMlpHidden + i] : __float2bfloat16(0.f);
    }
    for (int l = 0; l < kMlpLayers; ++l)
        for (int o = threadIdx.x; o < kMlpHidden; o += blockDim.x)
            S.bias[l][o] = o < mlp_out(l) ? params[mlp_w_offset(l) + mlp_in(l) * mlp_out(l) + o] : 0.f;
}

// acc[16 n-tiles][4] += A (16 x K, row-major in smem, stride lda) * W^T for
// W [128][K] in smem (stride ldw), K = 16 * ksteps.
__device__ __forceinline__ void gemm_rows_x_wT(float (*acc)[4], const __nv_bfloat16* A, int lda,
                                               const __nv_bfloat16* W, int ldw, int ksteps)
{
    const int lane = threadIdx.x & 31;
    for (int ks = 0; ks < ksteps; ++ks) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(a0, a1, a2, a3, A + (lane & 15) * lda + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int np = 0; np < 8; ++np) {
            uint32_t b0, b1, b2, b3;
            ldsm_x4(b0, b1, b2, b3,
                    W + (np * 16 + (lane & 7) + ((lane >> 4) << 3)) * ldw + ks * 16 + ((lane >> 3) & 1) * 8);
            mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
            mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
        }
    }
}

// ReLU(acc + bias) -> BF16 rows of the warp's next activation tile (and, when
// training, the global activation buffer).
__device__ __forceinline__ void store_hidden(float (*acc)[4], __nv_bfloat16* out, __nv_bfloat16* gout, int row0, int n)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = nt * 8 + t * 2;
        const uint32_t lo = pack_bf16(fmaxf(acc[nt][0], 0.f), fmaxf(acc[nt][1], 0.f));
        const uint32_t hi = pack_bf16(fmaxf(acc[nt][2], 0.f), fmaxf(acc[nt][3], 0.f));
        *reinterpret_cast<uint32_t*>(out + g * kPadH + col) = lo;
        *reinterpret_cast<uint32_t*>(out + (g + 8) * kPadH + col) = hi;
        if (gout) {
            if (row0 + g < n) *reinterpret_cast<uint32_t*>(gout + (size_t)(row0 + g) * kMlpHidden + col) = lo;
            if (row0 + g + 8 < n) *reinterpret_cast<uint32_t*>(gout + (size_t)(row0 + g + 8) * kMlpHidden + col) = hi;
        }
    }
}

__device__ __forceinline__ void init_acc(float (*acc)[4], const float* bias)
{
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const float b0 = bias[nt * 8 + t * 2], b1 = bias[nt * 8 + t * 2 + 1];
        acc[nt][0] = b0; acc[nt][1] = b1; acc[nt][2] = b0; acc[nt][3] = b1;
    }
}

// Forward of one 16-row tile already in S.act[warp][0] (cols 0..15); the
// output Y [16][4] (c layout) in y4.
__device__ __forceinline__ void forward_tile(FwdSmem& S, int warp, float* y4, __nv_bfloat16* gact, size_t act_stride,
                                             int row0, int n)
{
    float acc[16][4];
    __nv_bfloat16* bufA = S.act[warp][0];
    __nv_bfloat16* bufB = S.act[warp][1];
    init_acc(acc, S.bias[0]);
    gemm_rows_x_wT(acc, bufA, kPadH, S.w0, kPadIn, 1);
    store_hidden(acc, bufB, gact ? gact : nullptr, row0, n);
    __syncwarp();
    for (int l = 1; l <= 3; ++l) {
        init_acc(acc, S.bias[l]);
        gemm_rows_x_wT(acc, bufB, kPadH, S.w123[l - 1], kPadH, 8);
        __syncwarp();
        store_hidden(acc, bufA, gact ? gact + l * act_stride : nullptr, row0, n);
        __syncwarp();
        __nv_bfloat16* tmp = bufA; bufA = bufB; bufB = tmp;
    }
    // output layer (4 outputs padded to 8)
    const int lane = threadIdx.x & 31, t = lane & 3;
    float c[4];
    c[0] = t * 2 < kMlpOut ? S.bias[4][t * 2] : 0.f;
    c[1] = t * 2 + 1 < kMlpOut ? S.bias[4][t * 2 + 1] : 0.f;
    c[2] = c[0];
    c[3] = c[1];
    for (int ks = 0; ks < 8; ++ks) {
        uint32_t a0, a1, a2, a3, b0, b1;
        ldsm_x4(a0, a1, a2, a3, bufB + (lane & 15) * kPadH + ks * 16 + (lane >> 4) * 8);
        ldsm_x2(b0, b1, S.w4 + (lane & 7) * kPadH + ks * 16 + ((lane >> 3) & 1) * 8);
        mma16816(c, a0, a1, a2, a3, b0, b1);
    }
    y4[0] = c[0]; y4[1] = c[1]; y4[2] = c[2]; y4[3] = c[3];
}

}  // namespace mlpd
}  // namespace pivbos
