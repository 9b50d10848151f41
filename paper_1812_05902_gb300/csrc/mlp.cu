// MLP kernels of the surrogate (see mlp.cuh): inference and training on
// tcgen05 (mlp_tc.cuh, mlp_train_tc.cuh), Adam, and the warp-level BF16
// mma.sync m16n8k16 forward and backward (dX and dW per layer, ldmatrix
// operand loads from shared memory, FP32 accumulation) that PIVBOS_MLP_TC=0
// selects instead.
#include <math.h>
#include <stdlib.h>

#include "common.cuh"
#include "mlp.cuh"
#include "mlp_device.cuh"
#include "mlp_tc.cuh"
#include "mlp_train_tc.cuh"

namespace pivbos {
namespace {

using namespace mlpd;

__global__ void __launch_bounds__(kThreads, 1)
mlp_fwd_kernel(const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params,
               const __nv_bfloat16* __restrict__ X, int n, float* __restrict__ Y, __nv_bfloat16* __restrict__ gact,
               const float* __restrict__ T, __nv_bfloat16* __restrict__ dz, double* __restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
    load_network(S, wbf, params);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tiles = (n + 15) / 16;
    const size_t act_stride = (size_t)n * kMlpHidden;
    double lsum = 0.0;
    for (int tile = blockIdx.x * 8 + warp; tile < tiles; tile += gridDim.x * 8) {
        const int row0 = tile * 16;
        // input tile: 16 rows x 16 BF16 (32 B per row), two lanes per row
        {
            const int r = lane >> 1, h = lane & 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row0 + r < n) v = *reinterpret_cast<const uint4*>(X + (size_t)(row0 + r) * kMlpIn + h * 8);
            *reinterpret_cast<uint4*>(S.act[warp][0] + r * kPadH + h * 8) = v;
        }
        __syncwarp();
        float y4[4];
        forward_tile(S, warp, y4, gact, act_stride, row0, n);
        if (t * 2 < kMlpOut) {
            const int rows[2] = {row0 + g, row0 + g + 8};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = rows[h];
                if (r >= n) continue;
                const float ya = y4[2 * h], yb = y4[2 * h + 1];
                if (Y) {
                    Y[(size_t)r * kMlpOut + t * 2] = ya;
                    Y[(size_t)r * kMlpOut + t * 2 + 1] = yb;
                }
                if (T) {
                    const float da = ya - T[(size_t)r * kMlpOut + t * 2];
                    const float db = yb - T[(size_t)r * kMlpOut + t * 2 + 1];
                    lsum += (double)da * da + (double)db * db;
                    const float scale = 2.0f / ((float)n * kMlpOut);
                    *reinterpret_cast<uint32_t*>(dz + (size_t)r * kMlpHidden + t * 2) = pack_bf16(da * scale, db * scale);
                }
            }
        }
        if (T) {
            // zero the padding columns 4..15 of the output gradient rows
            const int r = lane >> 1, h = lane & 1;
            if (row0 + r < n) {
                __nv_bfloat16* p = dz + (size_t)(row0 + r) * kMlpHidden;
                if (h == 0) {
                    *reinterpret_cast<uint2*>(p + 4) = make_uint2(0, 0);
                } else {
                    *reinterpret_cast<uint4*>(p + 8) = make_uint4(0, 0, 0, 0);
                }
            }
        }
        __syncwarp();
    }
    if (loss) {
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum);
    }
}

// dZ_{l-1} = (dZ_l W_l) * (H_l > 0) for l >= 1.  dZ_l: [n][128] BF16 with
// valid columns out_l (4 -> zero padded to 16 for the output layer).
__global__ void __launch_bounds__(kThreads, 1)
mlp_dx_kernel(const __nv_bfloat16* __restrict__ wbf, int l, const __nv_bfloat16* __restrict__ dz_in, int n,
              const __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ dz_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int outl = mlp_out(l);
    const int kpad = outl < 16 ? 16 : outl;     // K of this product
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem_raw);            // [kpad][kPadH]
    __nv_bfloat16* Zs = Ws + kpad * kPadH;                                       // per warp [16][kPadH]
    for (int e = threadIdx.x; e < kpad * kMlpHidden; e += blockDim.x) {
        const int o = e / kMlpHidden, i = e % kMlpHidden;
        Ws[o * kPadH + i] = o < outl ? wbf[mlp_wbf_offset(l) + o * kMlpHidden + i] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __nv_bfloat16* Z = Zs + warp * 16 * kPadH;
    const int tiles = (n + 15) / 16;
    for (int tile = blockIdx.x * 8 + warp; tile < tiles; tile += gridDim.x * 8) {
        const int row0 = tile * 16;
        // stage dZ rows (kpad columns)
        for (int q = lane; q < 16 * (kpad / 8); q += 32) {
            const int r = q / (kpad / 8), c8 = q % (kpad / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row0 + r < n) v = *reinterpret_cast<const uint4*>(dz_in + (size_t)(row0 + r) * kMlpHidden + c8 * 8);
            *reinterpret_cast<uint4*>(Z + r * kPadH + c8 * 8) = v;
        }
        __syncwarp();
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        for (int ks = 0; ks < kpad / 16; ++ks) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, Z + (lane & 15) * kPadH + ks * 16 + (lane >> 4) * 8);
#pragma unroll
            for (int np = 0; np < 8; ++np) {
                // B (k = out, n = in) = W[out][in]: row-major K x N -> transposed loads
                const int mi = lane >> 3;
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(b0, b1, b2, b3,
                          Ws + (ks * 16 + (lane & 7) + (mi & 1) * 8) * kPadH + np * 16 + (mi >> 1) * 8);
                mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
                mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
            }
        }
        // mask by H_l > 0 and store
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int col = nt * 8 + t * 2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = row0 + g + h * 8;
                if (r >= n) continue;
                const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(H + (size_t)r * kMlpHidden + col);
                const float m0 = __bfloat162float(hv.x) > 0.f ? 1.f : 0.f;
                const float m1 = __bfloat162float(hv.y) > 0.f ? 1.f : 0.f;
                *reinterpret_cast<uint32_t*>(dz_out + (size_t)r * kMlpHidden + col) =
                    pack_bf16(acc[nt][2 * h] * m0, acc[nt][2 * h + 1] * m1);
            }
        }
        __syncwarp();
    }
}

// Partial dW_l = dZ_l^T H_l and db_l = sum dZ_l over the rows of this split.
// Warp w owns output rows [16w, 16w + 16).  H_l has in_l columns (row
// stride hstride).
__global__ void __launch_bounds__(kThreads, 1)
mlp_dw_kernel(int l, const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ H, int hstride, int n,
              int rows_per_split, float* __restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kRows = 64;   // rows staged per iteration
    const int outl = mlp_out(l), inl = mlp_in(l);
    const int mpad = outl < 16 ? 16 : outl;
    __nv_bfloat16* Zs = reinterpret_cast<__nv_bfloat16*>(smem_raw);   // [kRows][kPadH]
    __nv_bfloat16* Hs = Zs + kRows * kPadH;                           // [kRows][kPadH]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r_begin = blockIdx.x * rows_per_split;
    const int r_end = min(n, r_begin + rows_per_split);
    const int ntn = inl / 8;   // n-tiles (16 or 2)
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    float bsum = 0.f;   // db for output column threadIdx.x
    const bool active = warp * 16 < mpad;
    for (int r0 = r_begin; r0 < r_end; r0 += kRows) {
        __syncthreads();
        for (int q = threadIdx.x; q < kRows * (mpad / 8); q += blockDim.x) {
            const int r = q / (mpad / 8), c8 = q % (mpad / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + r < r_end) v = *reinterpret_cast<const uint4*>(dz + (size_t)(r0 + r) * kMlpHidden + c8 * 8);
            *reinterpret_cast<uint4*>(Zs + r * kPadH + c8 * 8) = v;
        }
        for (int q = threadIdx.x; q < kRows * (inl / 8); q += blockDim.x) {
            const int r = q / (inl / 8), c8 = q % (inl / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + r < r_end) v = *reinterpret_cast<const uint4*>(H + (size_t)(r0 + r) * hstride + c8 * 8);
            *reinterpret_cast<uint4*>(Hs + r * kPadH + c8 * 8) = v;
        }
        __syncthreads();
        if (threadIdx.x < outl)
            for (int r = 0; r < kRows; ++r) bsum += __bfloat162float(Zs[r * kPadH + threadIdx.x]);
        if (active) {
            for (int ks = 0; ks < kRows / 16; ++ks) {
                // A (m = out, k = row) = dZ^T: transposed loads of the dZ tile
                const int mi = lane >> 3;
                uint32_t a0, a1, a2, a3;
                ldsm_x4_t(a0, a1, a2, a3,
                          Zs + (ks * 16 + (lane & 7) + (mi >> 1) * 8) * kPadH + warp * 16 + (mi & 1) * 8);
                for (int np = 0; np < ntn / 2; ++np) {
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_t(b0, b1, b2, b3,
                              Hs + (ks * 16 + (lane & 7) + (mi & 1) * 8) * kPadH + np * 16 + (mi >> 1) * 8);
                    mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
                    mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
    }
    // partial sums of this split: [out][in] then [out]
    float* P = partial + (size_t)blockIdx.x * (outl * inl + outl);
    if (active) {
        for (int nt = 0; nt < ntn; ++nt) {
            const int col = nt * 8 + t * 2;
            const int ra = warp * 16 + g, rb = ra + 8;
            if (ra < outl) { P[ra * inl + col] = acc[nt][0]; P[ra * inl + col + 1] = acc[nt][1]; }
            if (rb < outl) { P[rb * inl + col] = acc[nt][2]; P[rb * inl + col + 1] = acc[nt][3]; }
        }
    }
    if (threadIdx.x < outl) P[outl * inl + threadIdx.x] = bsum;
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int splits, int count, float* __restrict__ grad)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float s = 0.f;
    for (int q = 0; q < splits; ++q) s += partial[(size_t)q * count + e];
    grad[e] = s;
}

// BF16 copies of parameter i = p: the weights [out][in] and, for layers 1-4,
// transposed [in][out] (the backward's operands).
__device__ __forceinline__ void store_bf16(int i, float p, __nv_bfloat16* __restrict__ wbf,
                                           __nv_bfloat16* __restrict__ wbfT)
{
    int l = 0;
    while (l + 1 < kMlpLayers && i >= mlp_w_offset(l + 1)) ++l;
    const int local = i - mlp_w_offset(l);
    if (local < mlp_in(l) * mlp_out(l)) {
        const __nv_bfloat16 b = __float2bfloat16(p);
        wbf[mlp_wbf_offset(l) + local] = b;
        if (l > 0 && wbfT) {
            const int o = local / mlp_in(l), j = local - o * mlp_in(l);
            wbfT[mlp_wbf_offset(l) + j * mlp_out(l) + o] = b;
        }
    }
}

__global__ void mlp_adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, __nv_bfloat16* __restrict__ wbf,
                                __nv_bfloat16* __restrict__ wbfT, float lr, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    p[i] = pi;
    store_bf16(i, pi, wbf, wbfT);
}

__global__ void mlp_tobf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ wbf,
                                  __nv_bfloat16* __restrict__ wbfT)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    store_bf16(i, p[i], wbf, wbfT);
}

// Inference forward on tcgen05: persistent CTAs of one warpgroup, one
// 128-row tile at a time, five MMA / epilogue rounds per tile; activations
// and accumulator in tensor memory (columns [0, 256)).
__global__ void __launch_bounds__(128, 1)
mlp_fwd_tc_kernel(const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params,
                  const __nv_bfloat16* __restrict__ X, int n, float* __restrict__ Y, int* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    mlptc::Net& S = *reinterpret_cast<mlptc::Net*>(smem);
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    mlptc::load_net(S, wbf, params);
    if (warp == 0) umma::tmem_alloc(&tmem_base, mlptc::kTileCols);
    if (tid == 0) {
        umma::mbar_init(&bar, 1);
        failed = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t d_tmem = tmem_base, a_tmem = tmem_base + mlptc::kACol;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    mlptc::store_constants(a_tmem + lane);
    uint32_t parity = 0;
    const int tiles = (n + mlptc::kRows - 1) / mlptc::kRows;
    for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
        const int row = t * mlptc::kRows + tid;
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
        if (row < n) {
            lo = *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn);
            hi = *reinterpret_cast<const uint4*>(X + (size_t)row * kMlpIn + 8);
        }
        mlptc::store_input(a_tmem + lane, lo, hi);
        // unrolled: each layer's descriptors and epilogue are fixed at compile time
#pragma unroll
        for (int l = 0; l < kMlpLayers; ++l) {
            umma::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                umma::fence_after_sync();
                mlptc::issue_layer(S, l, a_tmem, d_tmem);
                umma::commit(&bar);
                if (!umma::mbar_wait(&bar, parity, mlptc::kWaitLimit)) failed = 1;
            }
            __syncthreads();
            if (failed) break;
            parity ^= 1u;
            umma::fence_after_sync();
            if (l < kMlpLayers - 1) {
                mlptc::epilogue_hidden(d_tmem + lane, a_tmem + lane);
            } else {
                float y[kMlpOut];
                mlptc::epilogue_out(d_tmem + lane, y);
                if (row < n) *reinterpret_cast<float4*>(Y + (size_t)row * 4) = make_float4(y[0], y[1], y[2], y[3]);
            }
        }
    }
    if (failed && tid == 0) {
        // report, then give the MMAs in flight a second bounded wait before
        // the tensor memory is released
        atomicExch(status, (int)PIVBOS_ERR_DEVICE_TIMEOUT);
        umma::mbar_wait(&bar, parity, mlptc::kWaitLimit);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(tmem_base, mlptc::kTileCols);
    }
}

size_t tc_smem() { return sizeof(mlptc::Net); }

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

size_t dx_smem() { return (size_t)(kMlpHidden + 8 * 16) * kPadH * sizeof(__nv_bfloat16); }
size_t dw_smem() { return (size_t)2 * 64 * kPadH * sizeof(__nv_bfloat16); }

}  // namespace

cudaError_t mlp_alloc(MlpDev& d, int splits)
{
    d.splits = splits;
    cudaError_t e = cudaMalloc(&d.params, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&d.m, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&d.v, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&d.grad, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&d.wbf, sizeof(__nv_bfloat16) * kMlpWeights);
    if (e == cudaSuccess) e = cudaMalloc(&d.wbfT, sizeof(__nv_bfloat16) * kMlpWeights);
    if (e == cudaSuccess) e = cudaMalloc(&d.partial, sizeof(float) * (size_t)splits * (kMlpHidden * kMlpHidden + kMlpHidden));
    if (e == cudaSuccess) e = cudaMalloc(&d.status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d.m, 0, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(d.v, 0, sizeof(float) * kMlpParams);
    // the shared-memory limits are per device: set them on every allocation
    if (e == cudaSuccess) {
        e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FwdSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_dx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dx_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw_smem());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(mlptr::TrainSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_dw_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(mlptr::DwSmem));
    }
    return e;
}

void mlp_free(MlpDev& d)
{
    cudaFree(d.status);
    d.status = nullptr;
    cudaFree(d.params);
    cudaFree(d.m);
    cudaFree(d.v);
    cudaFree(d.grad);
    cudaFree(d.wbf);
    cudaFree(d.wbfT);
    cudaFree(d.partial);
    d = MlpDev();
}

cudaError_t mlp_work_alloc(MlpWork& w, int max_rows)
{
    w.max_rows = max_rows;
    cudaError_t e = cudaMalloc(&w.act, sizeof(__nv_bfloat16) * 4 * (size_t)max_rows * kMlpHidden);
    if (e == cudaSuccess)
        e = cudaMalloc(&w.dz, sizeof(__nv_bfloat16) * (4 * (size_t)max_rows * kMlpHidden +
                                                       (size_t)max_rows * mlptr::kDz4));
    if (e == cudaSuccess) e = cudaMalloc(&w.partial, sizeof(float) * (size_t)kMlpTcSplits * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&w.y, sizeof(float) * (size_t)max_rows * kMlpOut);
    if (e == cudaSuccess) e = cudaMalloc(&w.loss, sizeof(double));
    return e;
}

void mlp_work_free(MlpWork& w)
{
    cudaFree(w.act);
    cudaFree(w.dz);
    cudaFree(w.y);
    cudaFree(w.loss);
    cudaFree(w.partial);
    w = MlpWork();
}

cudaError_t mlp_sync_bf16(const MlpDev& d, cudaStream_t s)
{
    mlp_tobf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(d.params, d.wbf, d.wbfT);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_forward_tc(const MlpDev& d, const __nv_bfloat16* X, int n, float* Y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int tiles = (n + mlptc::kRows - 1) / mlptc::kRows;
    const int grid = min(sm_count(), tiles);
    timing_begin("mlp_forward_tc", s);
    mlp_fwd_tc_kernel<<<grid, 128, tc_smem(), s>>>(d.wbf, d.params, X, n, Y, d.status);
    timing_end("mlp_forward_tc", s);
    count_launches(1);
    return cudaGetLastError();
}

int mlp_status(const MlpDev& d)
{
    int v = 0;
    if (!d.status || cudaMemcpy(&v, d.status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    if (v) cudaMemset(d.status, 0, sizeof(int));
    return v;
}

static bool use_tc()
{
    static const bool v = [] {
        const char* e = getenv("PIVBOS_MLP_TC");
        return !(e && atoi(e) == 0);
    }();
    return v;
}

cudaError_t mlp_forward(const MlpDev& d, const __nv_bfloat16* X, int n, float* Y, MlpWork* work, const float* T,
                        cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (!work && use_tc()) return mlp_forward_tc(d, X, n, Y, s);
    if (work && use_tc()) {
        // the tcgen05 training forward; with targets also the loss and the
        // backward chain (mlp_backward then only forms the weight gradients)
        if (T) {
            cudaError_t e = cudaMemsetAsync(work->loss, 0, sizeof(double), s);
            if (e != cudaSuccess) return e;
        }
        const int tiles = (n + mlptc::kRows - 1) / mlptc::kRows;
        timing_begin("mlp_forward", s);
        mlp_train_tc_kernel<<<min(sm_count(), tiles), 128, sizeof(mlptr::TrainSmem), s>>>(
            d.wbf, d.wbfT, d.params, X, n, Y, T, work->act, work->dz, T ? work->loss : nullptr, d.status);
        timing_end("mlp_forward", s);
        count_launches(1);
        return cudaGetLastError();
    }
    const int tiles = (n + 15) / 16;
    const int grid = min(sm_count(), (tiles + 7) / 8);
    if (work && T) {
        cudaError_t e = cudaMemsetAsync(work->loss, 0, sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    timing_begin("mlp_forward", s);
    mlp_fwd_kernel<<<grid, kThreads, sizeof(FwdSmem), s>>>(d.wbf, d.params, X, n, Y, work ? work->act : nullptr, T,
                                                           work ? work->dz : nullptr,
                                                           (work && T) ? work->loss : nullptr);
    timing_end("mlp_forward", s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_backward(MlpDev& d, const __nv_bfloat16* X, int n, MlpWork& w, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (use_tc()) {
        // weight gradients of the five layers over row splits, then their sum
        const int chunks = (n + mlptc::kRows - 1) / mlptc::kRows;
        const int splits = min(kMlpTcSplits, chunks);
        const int rows_per_split = (chunks + splits - 1) / splits * mlptc::kRows;
        timing_begin("mlp_backward", s);
        mlp_dw_tc_kernel<<<dim3((unsigned)splits, kMlpLayers), 128, sizeof(mlptr::DwSmem), s>>>(
            X, w.act, w.dz, n, rows_per_split, w.partial, d.status);
        mlp_reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w.partial, splits, kMlpParams, d.grad);
        timing_end("mlp_backward", s);
        count_launches(2);
        return cudaGetLastError();
    }
    const int tiles = (n + 15) / 16;
    const int gx = min(sm_count(), (tiles + 7) / 8);
    const int rows_per_split = ((n + d.splits - 1) / d.splits + 15) / 16 * 16;
    const int splits = (n + rows_per_split - 1) / rows_per_split;
    const size_t act_stride = (size_t)n * kMlpHidden;
    int cur = 0;   // w.dz[cur] holds dZ of the current layer
    timing_begin("mlp_backward", s);
    for (int l = kMlpLayers - 1; l >= 0; --l) {
        const __nv_bfloat16* dzl = w.dz + (size_t)cur * w.max_rows * kMlpHidden;
        const __nv_bfloat16* Hl = l == 0 ? X : w.act + (size_t)(l - 1) * act_stride;
        const int hstride = l == 0 ? kMlpIn : kMlpHidden;
        mlp_dw_kernel<<<splits, kThreads, dw_smem(), s>>>(l, dzl, Hl, hstride, n, rows_per_split, d.partial);
        const int count = mlp_in(l) * mlp_out(l) + mlp_out(l);
        mlp_reduce_kernel<<<(count + 255) / 256, 256, 0, s>>>(d.partial, splits, count, d.grad + mlp_w_offset(l));
        count_launches(2);
        if (l > 0) {
            __nv_bfloat16* dzn = w.dz + (size_t)(1 - cur) * w.max_rows * kMlpHidden;
            mlp_dx_kernel<<<gx, kThreads, dx_smem(), s>>>(d.wbf, l, dzl, n, Hl, dzn);
            count_launches(1);
            cur = 1 - cur;
        }
    }
    timing_end("mlp_backward", s);
    return cudaGetLastError();
}

cudaError_t mlp_adam(MlpDev& d, int t, float lr, cudaStream_t s)
{
    // bias corrections in FP64: 1 - 0.999^t cancels (FP32 would lose ~2e-5
    // of it at small t)
    const float bc1 = (float)(1.0 - pow(0.9, (double)t));
    const float bc2 = (float)(1.0 - pow(0.999, (double)t));
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(d.params, d.m, d.v, d.grad, d.wbf, d.wbfT, lr, bc1,
                                                             bc2);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pivbos
