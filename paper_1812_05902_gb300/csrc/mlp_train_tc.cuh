// Training step of the surrogate network on the fifth-generation tensor
// cores (tcgen05), two kernels per step plus a reduction:
//
// 1. mlp_train_tc_kernel -- per 128-row tile, one warpgroup: the forward of
//    the five layers (as the inference kernel: weights in shared memory as
//    K-major operands, the biases carried through the MMA as BF16 leading
//    part and remainder), the loss and dL/dY, then the backward chain
//    dZ_{l-1} = (dZ_l W_l) * [H_{l-1} > 0] for l = 4..1 with the transposed
//    weights in shared memory.  The hidden activations stay in tensor
//    memory, where they are both the next layer's A operand and the ReLU
//    masks of the backward chain; the activations and the dZ's also go to
//    global memory for the weight gradients.  Activations and dZ are BF16,
//    every product accumulates in FP32.
// 2. mlp_dw_tc_kernel -- grid (splits, layer): dW_l = dZ_l^T H_{l-1} over a
//    split's rows, 128 rows (the K of the MMA) at a time staged transposed
//    into shared memory; the bias gradient rides along as a column of ones
//    in H (layer 0: its reserved input 14).  Layer 4 (4 outputs) is computed
//    transposed, dW_4^T = H_3^T dZ_4, so the 128 inputs fill the MMA's M;
//    its bias gradient is a block sum.  FP32 partial sums per split.
// 3. the reduction of the partial sums over the splits, in a fixed order
//    (mlp_reduce_kernel), then Adam.
//
// Tensor-memory columns of a tile (kernel 1): D [0, 128), the layer-0 input
// [128, 136), the inputs of layers 1-4 (H_0 .. H_3 with the two ones of the
// bias) 72 columns each from 136, the backward chain's A operand [424, 488).
#pragma once

#include <cuda_bf16.h>

#include "mlp.cuh"
#include "mlp_tc.cuh"
#include "umma.cuh"

namespace pivbos {
namespace mlptr {

using mlptc::kRows;
using mlptc::kKh;
using mlptc::kOutN;
using mlptc::kLboW;
using mlptc::kLboW4;
using mlptc::kOnes;
using mlptc::kWaitLimit;

constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColX = 128;                  // layer-0 input (8 columns)
constexpr uint32_t kColH = 136;                  // H_l at kColH + 72 l (72 columns each)
constexpr uint32_t kColHStride = 72;
constexpr uint32_t kColDz = 424;                 // backward A operand (64 columns)
constexpr int kDz4 = 16;                         // dZ_4 row stride (4 used)
constexpr uint32_t kLboT = (kMlpHidden / 8) * 128;   // K stride of a transposed weight operand (N = 128)

// Transposed weights W_l^T [N = in][K = out] of layers 1-4 (K-major), the
// backward chain's B operands; layer 4's K is padded from 4 to 16.
struct NetT {
    alignas(128) unsigned char wt[3][kMlpHidden * kMlpHidden * 2];
    alignas(128) unsigned char wt4[kMlpHidden * 16 * 2];
};

struct TrainSmem {
    mlptc::Net net;
    NetT nt;
};

// wbfT: per layer l >= 1 the BF16 weights transposed, [in][out] row-major.
__device__ inline void load_transposed(NetT& T, const __nv_bfloat16* __restrict__ wbfT)
{
    for (int l = 1; l <= 3; ++l) {
        for (int e = threadIdx.x; e < kMlpHidden * (kMlpHidden / 8); e += blockDim.x) {
            const int n = e / (kMlpHidden / 8), c = e % (kMlpHidden / 8);
            const uint4 v = *reinterpret_cast<const uint4*>(wbfT + mlp_wbf_offset(l) + n * kMlpHidden + c * 8);
            *reinterpret_cast<uint4*>(T.wt[l - 1] + umma::kmajor_offset(n, c * 8, kMlpHidden / 8)) = v;
        }
    }
    for (int e = threadIdx.x; e < kMlpHidden * 2; e += blockDim.x) {
        const int n = e >> 1, c = e & 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (c == 0) {   // the 4 outputs of input n; K 4..15 zero
            const uint2 w = *reinterpret_cast<const uint2*>(wbfT + mlp_wbf_offset(4) + n * kMlpOut);
            v.x = w.x;
            v.y = w.y;
        }
        *reinterpret_cast<uint4*>(T.wt4 + umma::kmajor_offset(n, c * 8, kMlpHidden / 8)) = v;
    }
}

__device__ __forceinline__ uint32_t mask_bf16x2(uint32_t d, uint32_t h)
{
    // keep each BF16 half of d where the activation's half is nonzero (the
    // ReLU output is positive exactly there)
    const uint32_t lo = (h & 0xffffu) ? 0xffffu : 0u, hi = (h >> 16) ? 0xffff0000u : 0u;
    return d & (lo | hi);
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

}  // namespace mlptr

// Kernel 1: forward, loss and the backward chain of 128-row tiles.
// act: H_0 .. H_3 [4][n][128] BF16; dz: dZ_0 .. dZ_3 [4][n][128] BF16 and
// dZ_4 [n][16] BF16 after them; Y [n][4] FP32 (may be null); T (targets
// [n][4], FP32) null: forward only.  loss: sum of squared errors (FP64).
__global__ void __launch_bounds__(128, 1)
mlp_train_tc_kernel(const __nv_bfloat16* __restrict__ wbf, const __nv_bfloat16* __restrict__ wbfT,
                    const float* __restrict__ params, const __nv_bfloat16* __restrict__ X, int n,
                    float* __restrict__ Y, const float* __restrict__ T, __nv_bfloat16* __restrict__ act,
                    __nv_bfloat16* __restrict__ dz, double* __restrict__ loss, int* __restrict__ status)
{
    using namespace mlptr;
    extern __shared__ __align__(128) unsigned char smem[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem);
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    mlptc::load_net(S.net, wbf, params);
    if (T) load_transposed(S.nt, wbfT);
    if (warp == 0) umma::tmem_alloc(&tmem_base, kTmemCols);
    if (tid == 0) {
        umma::mbar_init(&bar, 1);
        failed = 0;
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t d_t = tmem_base + lane;                 // this thread's row of D
    // the ones of the biases (and zeros up to K 144) of layers 1-4, once
    for (int l = 0; l < 4; ++l) mlptc::store_constants(tmem_base + kColH + kColHStride * l + lane);
    uint32_t parity = 0;
    double lsum = 0.0;
    const size_t plane = (size_t)n * kMlpHidden;
    const int tiles = (n + kRows - 1) / kRows;
    // one MMA chain, committed and waited for by thread 0; false if the wait gave up
    auto run = [&](auto issue) {
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            issue();
            umma::commit(&bar);
            if (!umma::mbar_wait(&bar, parity, kWaitLimit)) failed = 1;
        }
        __syncthreads();
        parity ^= 1u;
        umma::fence_after_sync();
        return !failed;
    };
    for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
        const int row = t * kRows + tid;
        const bool valid = row < n;
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
        if (valid) {
            lo = *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn);
            hi = *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn + 8);
        }
        mlptc::store_input(tmem_base + kColX + lane, lo, hi);
        // ---- forward
        bool ok = true;
#pragma unroll
        for (int l = 0; l < kMlpLayers && ok; ++l) {
            const uint32_t a_in = tmem_base + (l == 0 ? kColX : kColH + kColHStride * (l - 1));
            ok = run([&] { mlptc::issue_layer(S.net, l, a_in, tmem_base); });
            if (!ok) break;
            if (l < kMlpLayers - 1) {
                // H_l = ReLU(D) as BF16: the next layer's A, the mask, and global
                const uint32_t h_t = tmem_base + kColH + kColHStride * l + lane;
                uint32_t u[kMlpHidden];
#pragma unroll
                for (int c0 = 0; c0 < kMlpHidden; c0 += 32) umma::tmem_ld32_nowait(d_t + (uint32_t)c0, u + c0);
                umma::tmem_wait();
                uint32_t p[kMlpHidden / 2];
#pragma unroll
                for (int q = 0; q < kMlpHidden / 2; ++q)
                    p[q] = umma::relu_bf16x2(__uint_as_float(u[2 * q]), __uint_as_float(u[2 * q + 1]));
                umma::tmem_st32(h_t, p);
                umma::tmem_st32(h_t + 32, p + 32);
                if (valid && T) {
                    uint4* g = reinterpret_cast<uint4*>(act + (size_t)l * plane + (size_t)row * kMlpHidden);
#pragma unroll
                    for (int q = 0; q < kMlpHidden / 8; ++q)
                        g[q] = make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                }
                umma::tmem_wait_st();
            } else {
                float y[8];
                umma::tmem_ld8(d_t, y);
                if (valid && Y) *reinterpret_cast<float4*>(Y + (size_t)row * 4) = make_float4(y[0], y[1], y[2], y[3]);
                if (T) {
                    // dL/dY of the mean squared error over n x 4 outputs, as BF16
                    float d[4] = {0.f, 0.f, 0.f, 0.f};
                    if (valid) {
                        const float4 tt = *reinterpret_cast<const float4*>(T + (size_t)row * 4);
                        d[0] = y[0] - tt.x;
                        d[1] = y[1] - tt.y;
                        d[2] = y[2] - tt.z;
                        d[3] = y[3] - tt.w;
                        for (int c = 0; c < 4; ++c) lsum += (double)d[c] * d[c];
                    }
                    const float sc = 2.0f / ((float)n * kMlpOut);
                    const uint32_t q[8] = {bf16x2(d[0] * sc, d[1] * sc), bf16x2(d[2] * sc, d[3] * sc), 0u, 0u,
                                           0u, 0u, 0u, 0u};
                    umma::tmem_st8(tmem_base + kColDz + lane, q);
                    if (valid) {
                        uint4* g = reinterpret_cast<uint4*>(dz + 4 * plane + (size_t)row * kDz4);
                        g[0] = make_uint4(q[0], q[1], 0u, 0u);
                        g[1] = make_uint4(0u, 0u, 0u, 0u);
                    }
                    umma::tmem_wait_st();
                }
            }
        }
        if (!ok || !T) continue;
        // ---- backward chain: dZ_{l-1} from dZ_l, l = 4 .. 1
#pragma unroll
        for (int l = kMlpLayers - 1; l >= 1 && ok; --l) {
            ok = run([&] {
                const uint32_t w = umma::smem_addr(l == 4 ? S.nt.wt4 : S.nt.wt[l - 1]);
                const uint32_t idesc = umma::make_idesc_bf16(kRows, kMlpHidden);
                uint64_t bd = umma::make_desc(w, kLboT, 128);
                const int ksteps = l == 4 ? 1 : kMlpHidden / 16;
                for (int ks = 0; ks < ksteps; ++ks) {
                    umma::mma_bf16_ts(tmem_base, tmem_base + kColDz + 8 * ks, bd, idesc, ks > 0);
                    bd += (2 * kLboT) >> 4;
                }
            });
            if (!ok) break;
            uint32_t u[kMlpHidden], h[kMlpHidden / 2];
#pragma unroll
            for (int c0 = 0; c0 < kMlpHidden; c0 += 32) umma::tmem_ld32_nowait(d_t + (uint32_t)c0, u + c0);
            const uint32_t h_t = tmem_base + kColH + kColHStride * (l - 1) + lane;
            umma::tmem_ld32_nowait(h_t, h);
            umma::tmem_ld32_nowait(h_t + 32, h + 32);
            umma::tmem_wait();
            uint32_t p[kMlpHidden / 2];
#pragma unroll
            for (int q = 0; q < kMlpHidden / 2; ++q)
                p[q] = mask_bf16x2(bf16x2(__uint_as_float(u[2 * q]), __uint_as_float(u[2 * q + 1])), h[q]);
            if (l > 1) {
                umma::tmem_st32(tmem_base + kColDz + lane, p);
                umma::tmem_st32(tmem_base + kColDz + 32 + lane, p + 32);
            }
            if (valid) {
                uint4* g = reinterpret_cast<uint4*>(dz + (size_t)(l - 1) * plane + (size_t)row * kMlpHidden);
#pragma unroll
                for (int q = 0; q < kMlpHidden / 8; ++q)
                    g[q] = make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
            }
            if (l > 1) umma::tmem_wait_st();
        }
    }
    if (loss) {
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if ((tid & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum);
    }
    if (failed && tid == 0) {
        // report, then give the MMAs in flight a second bounded wait before
        // the tensor memory is released
        atomicExch(status, (int)PIVBOS_ERR_DEVICE_TIMEOUT);
        umma::mbar_wait(&bar, parity, kWaitLimit);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Kernel 2: weight (and bias) gradients of one layer (blockIdx.y) over the
// rows of one split (blockIdx.x), FP32 partial sums [split][kMlpParams].
namespace mlptr {

constexpr int kDwN = 144;   // N of layers 0-3's dW MMA: inputs, the ones column, zeros

struct DwSmem {
    alignas(128) unsigned char a[kRows * kMlpHidden * 2];   // A [M = 128][K = 128 rows]
    alignas(128) unsigned char b[kDwN * kRows * 2];          // B [N <= 144][K = 128 rows]
};

__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t off, uint16_t v)
{
    *reinterpret_cast<uint16_t*>(base + off) = v;
}

}  // namespace mlptr

__global__ void __launch_bounds__(128, 1)
mlp_dw_tc_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ act,
                 const __nv_bfloat16* __restrict__ dz, int n, int rows_per_split, float* __restrict__ partial,
                 int* __restrict__ status)
{
    using namespace mlptr;
    extern __shared__ __align__(128) unsigned char smem[];
    DwSmem& S = *reinterpret_cast<DwSmem*>(smem);
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    __shared__ float bsum[4][kMlpOut];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int l = blockIdx.y;
    const int in = mlp_in(l), out = mlp_out(l);
    // layer 4 is taken transposed: M = its 128 inputs, N = its outputs (16)
    const int N = l == 4 ? 16 : (l == 0 ? kMlpIn : kDwN);
    if (warp == 0) umma::tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        umma::mbar_init(&bar, 1);
        failed = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const size_t plane = (size_t)n * kMlpHidden;
    const int r0 = blockIdx.x * rows_per_split, r1 = min(n, r0 + rows_per_split);
    const __nv_bfloat16* dzl = dz + (size_t)l * plane;
    const __nv_bfloat16* hin = l == 0 ? X : act + (size_t)(l - 1) * plane;
    const uint16_t one = 0x3F80u;
    float db4[kMlpOut] = {0.f, 0.f, 0.f, 0.f};
    uint32_t parity = 0;
    int chunks = 0;
    for (int c0 = r0; c0 < r1 && !failed; c0 += kRows, ++chunks) {
        // Staging: thread k loads row c0 + k of each operand with 16-byte
        // loads and scatters it into the K-major layout as column k.
        const int row = c0 + tid;
        const bool valid = row < r1;
        const uint32_t k = (uint32_t)tid;   // this row's K index within the chunk
        // 128 BF16 of a row (zeros past the split's rows)
        auto load128 = [&](const __nv_bfloat16* src, uint32_t* v) {
#pragma unroll
            for (int q = 0; q < kMlpHidden / 8; ++q) {
                const uint4 w = valid ? *reinterpret_cast<const uint4*>(src + (size_t)row * kMlpHidden + 8 * q)
                                      : make_uint4(0u, 0u, 0u, 0u);
                v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
            }
        };
        auto scatter128 = [&](unsigned char* dst, int groups, const uint32_t* v) {
#pragma unroll
            for (int m = 0; m < kMlpHidden; ++m)
                st_bf16(dst, umma::kmajor_offset(m, k, groups), (uint16_t)(v[m >> 1] >> (16 * (m & 1))));
        };
        uint32_t v[kMlpHidden / 2];
        if (l < 4) {
            // A = dZ_l^T: element (m = output, k = row)
            load128(dzl, v);
            scatter128(S.a, kRows / 8, v);
            if (l > 0) {
                // B = [H_{l-1} | 1]^T: element (n = input, k = row), the
                // ones in column 128, zeros to 143
                load128(hin, v);
                scatter128(S.b, kDwN / 8, v);
#pragma unroll
                for (int j = kMlpHidden; j < kDwN; ++j)
                    st_bf16(S.b, umma::kmajor_offset(j, k, kDwN / 8), (valid && j == kMlpHidden) ? one : (uint16_t)0);
            } else {
                // layer 0: the 16 inputs, the reserved input 14 carrying the ones
                const uint4 lo = valid ? *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn) : make_uint4(0u, 0u, 0u, 0u);
                const uint4 hi = valid ? *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn + 8)
                                       : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t xv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                for (int j = 0; j < kMlpIn; ++j) {
                    uint16_t b = (uint16_t)(xv[j >> 1] >> (16 * (j & 1)));
                    if (j == kMlpIn - 2) b = valid ? one : (uint16_t)0;
                    if (j == kMlpIn - 1) b = 0;
                    st_bf16(S.b, umma::kmajor_offset(j, k, kMlpIn / 8), b);
                }
            }
        } else {
            // A = H_3^T: element (m = input, k = row); B = dZ_4^T (n = output,
            // 4 of 16), whose sums over the rows are the output bias's gradient
            load128(hin, v);
            scatter128(S.a, kRows / 8, v);
            const uint2 d = valid ? *reinterpret_cast<const uint2*>(dz + 4 * plane + (size_t)row * kDz4)
                                  : make_uint2(0u, 0u);
            const uint16_t dd[4] = {(uint16_t)(d.x & 0xffffu), (uint16_t)(d.x >> 16), (uint16_t)(d.y & 0xffffu),
                                    (uint16_t)(d.y >> 16)};
#pragma unroll
            for (int j = 0; j < 16; ++j) st_bf16(S.b, umma::kmajor_offset(j, k, 2), j < 4 ? dd[j] : (uint16_t)0);
#pragma unroll
            for (int c = 0; c < 4; ++c) db4[c] += __bfloat162float(__ushort_as_bfloat16(dd[c]));
        }
        umma::fence_async_smem();
        umma::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t idesc = umma::make_idesc_bf16(kRows, N);
            uint64_t ad = umma::make_desc(umma::smem_addr(S.a), (kRows / 8) * 128, 128);
            uint64_t bd = umma::make_desc(umma::smem_addr(S.b), (uint32_t)(N / 8) * 128, 128);
            for (int ks = 0; ks < kRows / 16; ++ks) {
                umma::mma_bf16(tmem_base, ad, bd, idesc, chunks > 0 || ks > 0);
                ad += (2 * (kRows / 8) * 128) >> 4;
                bd += (2 * (uint32_t)(N / 8) * 128) >> 4;
            }
            umma::commit(&bar);
            if (!umma::mbar_wait(&bar, parity, kWaitLimit)) failed = 1;
        }
        __syncthreads();   // the next chunk overwrites the operands
        parity ^= 1u;
        umma::fence_after_sync();
    }
    // partial sums of this split
    float* P = partial + (size_t)blockIdx.x * kMlpParams + mlp_w_offset(l);
    const int m = tid;   // this thread's TMEM lane: an output (layers 0-3) or an input (layer 4)
    const uint32_t d_t = tmem_base + ((uint32_t)(warp * 32) << 16);
    if (!failed) {
        float v[kDwN];
        if (chunks > 0) {
            for (int c0 = 0; c0 < N; c0 += 16) {
                float w8[8];
                umma::tmem_ld8(d_t + (uint32_t)c0, w8);
                for (int q = 0; q < 8; ++q) v[c0 + q] = w8[q];
                umma::tmem_ld8(d_t + (uint32_t)c0 + 8, w8);
                for (int q = 0; q < 8; ++q) v[c0 + 8 + q] = w8[q];
            }
        } else {
            for (int q = 0; q < N; ++q) v[q] = 0.f;
        }
        if (l < 4) {
            for (int j = 0; j < in; ++j) P[m * in + j] = (l == 0 && j >= kMlpIn - 2) ? 0.f : v[j];
            P[out * in + m] = v[l == 0 ? kMlpIn - 2 : kMlpHidden];
        } else {
            for (int c = 0; c < kMlpOut; ++c) P[c * kMlpHidden + m] = v[c];
        }
    }
    if (l == 4) {
        // the output bias: the sum of dZ_4 over the split's rows, in a fixed order
        for (int c = 0; c < kMlpOut; ++c)
            for (int off = 16; off > 0; off >>= 1) db4[c] += __shfl_xor_sync(0xffffffffu, db4[c], off);
        if ((tid & 31) == 0)
            for (int c = 0; c < kMlpOut; ++c) bsum[warp][c] = db4[c];
        __syncthreads();
        if (tid < kMlpOut) P[kMlpOut * kMlpHidden + tid] = bsum[0][tid] + bsum[1][tid] + bsum[2][tid] + bsum[3][tid];
    }
    if (failed && tid == 0) {
        atomicExch(status, (int)PIVBOS_ERR_DEVICE_TIMEOUT);
        umma::mbar_wait(&bar, parity, kWaitLimit);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem_base, 256);
    }
}

}  // namespace pivbos
