// Medium preparation (Sec. 3.2): Gladstone-Dale (Eq. 1) and the node
// gradient of n that Eq. 6 samples, packed as one float4 per node.
#include "common.cuh"

namespace pivbos {

// Derivative along one axis from three node densities around position q of
// N nodes: central difference inside, second-order one-sided at the ends,
// two-point difference when the axis has two nodes.  Differences of rho are
// taken before scaling so that nearly equal densities subtract exactly.
__device__ __forceinline__ float axis_diff(const float* __restrict__ rho, int base, int stride, int q,
                                           int N, float k_over_2h)
{
    if (N == 2) {
        // nodes q = 0 and q = 1 both take (f1 - f0) / h
        const int b0 = base - q * stride;
        return (__ldg(rho + b0 + stride) - __ldg(rho + b0)) * (2.0f * k_over_2h);
    }
    if (q == 0) {
        const float f0 = __ldg(rho + base), f1 = __ldg(rho + base + stride), f2 = __ldg(rho + base + 2 * stride);
        return (4.0f * (f1 - f0) - (f2 - f0)) * k_over_2h;
    }
    if (q == N - 1) {
        const float f0 = __ldg(rho + base), f1 = __ldg(rho + base - stride), f2 = __ldg(rho + base - 2 * stride);
        return -(4.0f * (f1 - f0) - (f2 - f0)) * k_over_2h;
    }
    return (__ldg(rho + base + stride) - __ldg(rho + base - stride)) * k_over_2h;
}

__global__ void medium_prep_kernel(const float* __restrict__ rho, float4* __restrict__ field, int nx, int ny,
                                   int nz, float K, float kx, float ky, float kz)
{
    const int64_t total = (int64_t)nx * ny * nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += stride) {
        const int i = (int)(p % nx);
        const int j = (int)((p / nx) % ny);
        const int k = (int)(p / ((int64_t)nx * ny));
        const int base = (int)p;
        float4 v;
        v.x = K * __ldg(rho + base);
        v.y = axis_diff(rho, base, 1, i, nx, kx);
        v.z = axis_diff(rho, base, nx, j, ny, ky);
        v.w = axis_diff(rho, base, nx * ny, k, nz, kz);
        field[p] = v;
    }
}

cudaError_t launch_medium_prep(const float* rho, float4* field, int nx, int ny, int nz,
                               const double spacing[3], double K, cudaStream_t s)
{
    const int64_t total = (int64_t)nx * ny * nz;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    const float kx = (float)(K / (2.0 * spacing[0]));
    const float ky = (float)(K / (2.0 * spacing[1]));
    const float kz = (float)(K / (2.0 * spacing[2]));
    timing_begin("medium_prep", s);
    medium_prep_kernel<<<(unsigned)blocks, 256, 0, s>>>(rho, field, nx, ny, nz, (float)K, kx, ky, kz);
    timing_end("medium_prep", s);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pivbos
