// Source ordering (Sec. 3.5 groups the rays of one source in one block):
// sources are sorted along a Morton (Z-order) curve of their (x, y) so that
// consecutive CTAs trace neighbouring sources, whose rays cross the same part
// of the density grid and land on the same part of the sensor.
//
// Keys: 16 bits per axis over [-1 m, 1 m) (clamped), interleaved, in the
// high 32 bits; the source index in the low 32 bits (so keys are unique).
// The last pass writes the permutation and the sorted source positions as
// double-float pairs, the form the tracer reads.
// Sort: bitonic network over the next power of two, with all strides below
// kSortBlock elements done in shared memory.
#include "common.cuh"

namespace pivbos {

constexpr int kSortThreads = 512;
constexpr int kSortBlock = 2 * kSortThreads;   // elements per shared-memory block

__device__ __forceinline__ uint32_t spread16(uint32_t v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void morton_keys_kernel(const double* __restrict__ src, uint32_t n, uint32_t n_pow2,
                                   uint64_t* __restrict__ keys)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pow2) return;
    if (q >= n) {
        keys[q] = ~0ull;
        return;
    }
    const double x = src[3 * (size_t)q], y = src[3 * (size_t)q + 1];
    const double fx = fmin(fmax((x + 1.0) * 32768.0, 0.0), 65535.0);
    const double fy = fmin(fmax((y + 1.0) * 32768.0, 0.0), 65535.0);
    const uint32_t code = spread16((uint32_t)fx) | (spread16((uint32_t)fy) << 1);
    keys[q] = ((uint64_t)code << 32) | q;
}

__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b, bool up)
{
    if ((a > b) == up) {
        const uint64_t t = a;
        a = b;
        b = t;
    }
}

// Full sort of each kSortBlock-element block (stages k = 2 .. min(n, kSortBlock)),
// or, with merge_k > 0, the strides j < kSortBlock of stage merge_k.
__global__ void bitonic_shared_kernel(uint64_t* __restrict__ keys, uint32_t n_pow2, uint32_t merge_k)
{
    __shared__ uint64_t s[kSortBlock];
    const uint32_t base = blockIdx.x * kSortBlock;
    const uint32_t len = min((uint32_t)kSortBlock, n_pow2);
    for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) s[q] = keys[base + q];
    __syncthreads();
    const uint32_t k_lo = merge_k ? merge_k : 2;
    const uint32_t k_hi = merge_k ? merge_k : len;
    for (uint32_t k = k_lo; k <= k_hi; k <<= 1) {
        for (uint32_t j = min(k >> 1, len >> 1); j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < len / 2; t += blockDim.x) {
                // t-th pair of this stride: i has bit j clear
                const uint32_t i = 2 * t - (t & (j - 1));
                const uint32_t l = i + j;
                const bool up = ((base + i) & k) == 0;
                uint64_t a = s[i], b = s[l];
                cmp_swap(a, b, up);
                s[i] = a;
                s[l] = b;
            }
            __syncthreads();
        }
    }
    for (uint32_t q = threadIdx.x; q < len; q += blockDim.x) keys[base + q] = s[q];
}

__global__ void bitonic_global_kernel(uint64_t* __restrict__ keys, uint32_t n_pow2, uint32_t j, uint32_t k)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pow2 / 2) return;
    const uint32_t i = 2 * t - (t & (j - 1));
    const uint32_t l = i + j;
    const bool up = (i & k) == 0;
    uint64_t a = keys[i], b = keys[l];
    cmp_swap(a, b, up);
    keys[i] = a;
    keys[l] = b;
}

__global__ void keys_to_perm_kernel(const uint64_t* __restrict__ keys, const double* __restrict__ src, uint32_t n,
                                    uint32_t* __restrict__ perm, float2* __restrict__ src_df)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t sid = (uint32_t)keys[q];
    perm[q] = sid;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = src[3 * (size_t)sid + a];
        const float hi = __double2float_rn(v);
        src_df[3 * (size_t)q + a] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

cudaError_t launch_morton_sort(const double* sources, uint32_t n, uint64_t* keys, uint32_t n_pow2,
                               uint32_t* perm, float2* src_df, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    timing_begin("sort", s);
    int64_t launched = 3;
    morton_keys_kernel<<<(n_pow2 + 255) / 256, 256, 0, s>>>(sources, n, n_pow2, keys);
    const uint32_t blocks = (n_pow2 + kSortBlock - 1) / kSortBlock;
    bitonic_shared_kernel<<<blocks, kSortThreads, 0, s>>>(keys, n_pow2, 0);
    for (uint32_t k = 2 * kSortBlock; k <= n_pow2; k <<= 1) {
        for (uint32_t j = k >> 1; j >= (uint32_t)kSortBlock; j >>= 1)
        {
            bitonic_global_kernel<<<(n_pow2 / 2 + 255) / 256, 256, 0, s>>>(keys, n_pow2, j, k);
            ++launched;
        }
        bitonic_shared_kernel<<<blocks, kSortThreads, 0, s>>>(keys, n_pow2, k);
        ++launched;
    }
    keys_to_perm_kernel<<<(n + 255) / 256, 256, 0, s>>>(keys, sources, n, perm, src_df);
    timing_end("sort", s);
    count_launches(launched);
    return cudaGetLastError();
}

}  // namespace pivbos
