// The surrogate network's forward pass on the fifth-generation tensor cores:
// 128-row tiles, weights resident in shared memory as K-major core-matrix
// operands, one 128 x 128 (or 128 x 16) FP32 accumulator per layer in
// tensor memory, and an epilogue (bias, ReLU, BF16) from tensor memory back
// into the next layer's shared-memory operand.  One warpgroup (4 warps)
// owns a tile: warp w reads accumulator lanes (rows) 32w .. 32w + 31.
#pragma once

#include <cuda_bf16.h>

#include "mlp.cuh"
#include "umma.cuh"

namespace pivbos {
namespace mlptc {

constexpr int kRows = 128;                                 // rows per tile (MMA M)
constexpr int kGroups = kRows / 8;                         // row groups of an A tile
constexpr uint32_t kTileBytes = kRows * kMlpHidden * 2;    // A operand of one tile (K up to 128)
constexpr int kOutN = 16;                                  // output layer N (4 used)
constexpr uint32_t kLboA = kGroups * 128;                  // K-direction core-matrix stride of A
constexpr uint32_t kLboW = (kMlpHidden / 8) * 128;         // the same for a 128-row weight matrix
constexpr uint32_t kLboW4 = (kOutN / 8) * 128;             // ... and for the 16-row output weights
constexpr uint32_t kWaitLimit = 1u << 20;                  // mbarrier polls before giving up

struct Net {
    alignas(128) unsigned char w0[kMlpHidden * kMlpIn * 2];
    alignas(128) unsigned char wh[3][kMlpHidden * kMlpHidden * 2];
    alignas(128) unsigned char w4[kOutN * kMlpHidden * 2];
    float bias[4][kMlpHidden];
    float bias4[kOutN];
};

// Weights (BF16 [out][in] per layer in wbf) and biases (FP32 master) into
// shared memory, 16 bytes at a time.
__device__ inline void load_net(Net& S, const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params)
{
    for (int e = threadIdx.x; e < kMlpHidden * (kMlpIn / 8); e += blockDim.x) {
        const int n = e / (kMlpIn / 8), c = e % (kMlpIn / 8);
        *reinterpret_cast<uint4*>(S.w0 + umma::kmajor_offset(n, c * 8, kMlpHidden / 8)) =
            *reinterpret_cast<const uint4*>(wbf + mlp_wbf_offset(0) + n * kMlpIn + c * 8);
    }
    for (int l = 1; l <= 3; ++l)
        for (int e = threadIdx.x; e < kMlpHidden * (kMlpHidden / 8); e += blockDim.x) {
            const int n = e / (kMlpHidden / 8), c = e % (kMlpHidden / 8);
            *reinterpret_cast<uint4*>(S.wh[l - 1] + umma::kmajor_offset(n, c * 8, kMlpHidden / 8)) =
                *reinterpret_cast<const uint4*>(wbf + mlp_wbf_offset(l) + n * kMlpHidden + c * 8);
        }
    for (int e = threadIdx.x; e < kOutN * (kMlpHidden / 8); e += blockDim.x) {
        const int n = e / (kMlpHidden / 8), c = e % (kMlpHidden / 8);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (n < kMlpOut) v = *reinterpret_cast<const uint4*>(wbf + mlp_wbf_offset(4) + n * kMlpHidden + c * 8);
        *reinterpret_cast<uint4*>(S.w4 + umma::kmajor_offset(n, c * 8, kOutN / 8)) = v;
    }
    for (int e = threadIdx.x; e < 4 * kMlpHidden; e += blockDim.x) {
        const int l = e / kMlpHidden, o = e % kMlpHidden;
        S.bias[l][o] = params[mlp_w_offset(l) + mlp_in(l) * mlp_out(l) + o];
    }
    for (int o = threadIdx.x; o < kOutN; o += blockDim.x)
        S.bias4[o] = o < kMlpOut ? params[mlp_w_offset(4) + kMlpHidden * kMlpOut + o] : 0.0f;
}

// Row r of the input tile: 16 BF16 features.
__device__ __forceinline__ void store_input_row(unsigned char* A, int r, uint4 lo, uint4 hi)
{
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, 0, kGroups)) = lo;
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, 8, kGroups)) = hi;
}

// Issue layer l of one tile (one thread): D[tmem] = A * W_l^T.
__device__ __forceinline__ void issue_layer(const Net& S, int l, uint32_t a_saddr, uint32_t d_tmem)
{
    if (l == 0) {
        umma::mma_bf16(d_tmem, umma::make_desc(a_saddr, kLboA, 128),
                       umma::make_desc(umma::smem_addr(S.w0), kLboW, 128), umma::make_idesc_bf16(kRows, kMlpHidden),
                       false);
        return;
    }
    const uint32_t w = l < 4 ? umma::smem_addr(S.wh[l - 1]) : umma::smem_addr(S.w4);
    const uint32_t lbo_w = l < 4 ? kLboW : kLboW4;
    const uint32_t idesc = umma::make_idesc_bf16(kRows, l < 4 ? kMlpHidden : kOutN);
    // successive K steps advance both start addresses by two core matrices
    // along K: add (2 * LBO) >> 4 to the descriptors' address fields
    uint64_t ad = umma::make_desc(a_saddr, kLboA, 128);
    uint64_t bd = umma::make_desc(w, lbo_w, 128);
    const uint64_t ainc = (2 * kLboA) >> 4, binc = (2 * lbo_w) >> 4;
#pragma unroll
    for (int ks = 0; ks < kMlpHidden / 16; ++ks) {
        umma::mma_bf16(d_tmem, ad, bd, idesc, ks > 0);
        ad += ainc;
        bd += binc;
    }
}

// Hidden-layer epilogue of this thread's row r: ReLU(D + b) as BF16 into the
// next layer's A operand.
__device__ __forceinline__ void epilogue_hidden(uint32_t row_tmem, const float* __restrict__ bias, unsigned char* A,
                                                int r)
{
#pragma unroll 1
    for (int c0 = 0; c0 < kMlpHidden; c0 += 32) {
        float v[32];
        umma::tmem_ld32(row_tmem + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t p[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = j * 8 + q * 2;
                const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[i] + bias[c0 + i], 0.0f),
                                                               fmaxf(v[i + 1] + bias[c0 + i + 1], 0.0f));
                p[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
            *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, c0 + j * 8, kGroups)) =
                make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// The same with two 32-column loads in flight per wait and the ReLU folded
// into the BF16 conversion.
__device__ __forceinline__ void epilogue_hidden2(uint32_t row_tmem, const float* __restrict__ bias, unsigned char* A,
                                                 int r)
{
#pragma unroll 1
    for (int c0 = 0; c0 < kMlpHidden; c0 += 64) {
        uint32_t u[64];
        umma::tmem_ld32_nowait(row_tmem + (uint32_t)c0, u);
        umma::tmem_ld32_nowait(row_tmem + (uint32_t)c0 + 32, u + 32);
        umma::tmem_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t p[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = j * 8 + q * 2;
                p[q] = umma::relu_bf16x2(__uint_as_float(u[i]) + bias[c0 + i],
                                         __uint_as_float(u[i + 1]) + bias[c0 + i + 1]);
            }
            *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, c0 + j * 8, kGroups)) =
                make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// Output epilogue: the 4 outputs of this thread's row.
__device__ __forceinline__ void epilogue_out(uint32_t row_tmem, const float* __restrict__ bias4, float* y)
{
    float v[8];
    umma::tmem_ld8(row_tmem, v);
#pragma unroll
    for (int c = 0; c < kMlpOut; ++c) y[c] = v[c] + bias4[c];
}

}  // namespace mlptc
}  // namespace pivbos
