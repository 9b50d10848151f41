// Image pairs for displacement analysis and 16-bit images: the second
// frame's particles moved by a velocity field, and the 32.32 image converted
// to the 16 bits a camera writes (Sec. 3.4: ~1e4 rays per particle give a
// 16-bit dynamic range).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>

#include "handles.cuh"

namespace pivbos {

struct VelGrid {
    const float* v;   // [nz][ny][nx][3]
    int n[3];
    double origin[3], h[3];
};

// trilinear sample of the velocity, the point clamped into the grid (FP64)
__device__ __forceinline__ void vel_sample(const VelGrid& G, const double x[3], double u[3])
{
    int c[3];
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double g = fmin(fmax((x[a] - G.origin[a]) / G.h[a], 0.0), (double)(G.n[a] - 1));
        c[a] = min((int)g, G.n[a] - 2);
        f[a] = g - (double)c[a];
    }
    u[0] = u[1] = u[2] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int di = q & 1, dj = (q >> 1) & 1, dk = q >> 2;
        const double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        const float* p = G.v + 3 * (((size_t)(c[2] + dk) * G.n[1] + (c[1] + dj)) * G.n[0] + (c[0] + di));
        u[0] += w * (double)__ldg(p);
        u[1] += w * (double)__ldg(p + 1);
        u[2] += w * (double)__ldg(p + 2);
    }
}

// explicit midpoint rule: k = u(x), x' = x + dt u(x + dt k / 2); one thread per particle
__global__ void advect_kernel(const VelGrid G, const double* __restrict__ src, int64_t n, double dt,
                              double* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double x[3] = {src[3 * q], src[3 * q + 1], src[3 * q + 2]};
    double k[3], u[3];
    vel_sample(G, x, k);
    const double xm[3] = {x[0] + 0.5 * dt * k[0], x[1] + 0.5 * dt * k[1], x[2] + 0.5 * dt * k[2]};
    vel_sample(G, xm, u);
    out[3 * q] = x[0] + dt * u[0];
    out[3 * q + 1] = x[1] + dt * u[1];
    out[3 * q + 2] = x[2] + dt * u[2];
}

// counts = (image + floor(d/2)) / d (integer division), clipped to
// [0, 65535]; d = llround(full_scale 2^32 / 65535) >= 1, thr = 65535 d -
// floor(d/2) (counts reach 65535 from there).  The quotient is at most 65535:
// an FP32 estimate from the reciprocal of d is within one of it, and one
// exact 64-bit multiply-subtract corrects it, so no FP64 or 64-bit division
// runs per pixel.
struct U16Scale {
    long long d, h, thr;
    float inv_d;
};

__device__ __forceinline__ uint32_t to_u16(long long v, const U16Scale& S)
{
    if (v <= 0) return 0u;
    if (v >= S.thr) return 65535u;
    const unsigned long long x = (unsigned long long)(v + S.h);
    const float xf = fmaf((float)(uint32_t)(x >> 32), 4294967296.0f, (float)(uint32_t)x);
    long long q = (int)(xf * S.inv_d);   // below 65536: a 32-bit conversion
    const long long r = (long long)x - q * S.d;
    q += (r >= S.d) - (r < 0);
    return (uint32_t)q;
}

// 8 pixels per thread and step: 64 B read as four 16-byte loads, 16 B written
// as one; grid-stride over the image (the host sizes the grid to the SMs).
__global__ void image_u16_kernel(const int64_t* __restrict__ img, int64_t n, const U16Scale S,
                                 uint16_t* __restrict__ out)
{
    const int64_t n8 = n / 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const longlong2* in2 = reinterpret_cast<const longlong2*>(img);
    uint4* out8 = reinterpret_cast<uint4*>(out);
    for (int64_t t = t0; t < n8; t += stride) {
        const longlong2 a = __ldcs(in2 + 4 * t), b = __ldcs(in2 + 4 * t + 1);
        const longlong2 c = __ldcs(in2 + 4 * t + 2), d = __ldcs(in2 + 4 * t + 3);
        uint4 o;
        o.x = to_u16(a.x, S) | (to_u16(a.y, S) << 16);
        o.y = to_u16(b.x, S) | (to_u16(b.y, S) << 16);
        o.z = to_u16(c.x, S) | (to_u16(c.y, S) << 16);
        o.w = to_u16(d.x, S) | (to_u16(d.y, S) << 16);
        __stcs(out8 + t, o);
    }
    for (int64_t q = 8 * n8 + t0; q < n; q += stride) out[q] = (uint16_t)to_u16(img[q], S);
}

}  // namespace pivbos


extern "C" {

pivbos_status pivbos_advect_sources(const double* sources, int64_t n_sources, const float* velocity, int nx, int ny,
                                    int nz, const double origin[3], const double spacing[3], double dt,
                                    double* out, void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (n_sources < 0 || n_sources > (1ll << 31)) return failf(PIVBOS_ERR_INVALID_ARG, "n_sources");
    if (nx < 2 || ny < 2 || nz < 2 || !origin || !spacing || !isfinite(dt))
        return failf(PIVBOS_ERR_INVALID_ARG, "grid or dt");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(origin[a]) || !(spacing[a] > 0.0) || !isfinite(spacing[a]))
            return failf(PIVBOS_ERR_INVALID_ARG, "origin or spacing");
    if (n_sources == 0) return PIVBOS_OK;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return failf(PIVBOS_ERR_CUDA, "cudaGetDevice");
    }
    pivbos_status st;
    if ((st = device_pointer(sources, dev, "sources")) || (st = device_pointer(velocity, dev, "velocity")) ||
        (st = device_pointer(out, dev, "out")))
        return st;
    VelGrid G;
    G.v = velocity;
    G.n[0] = nx;
    G.n[1] = ny;
    G.n[2] = nz;
    for (int a = 0; a < 3; ++a) {
        G.origin[a] = origin[a];
        G.h[a] = spacing[a];
    }
    cudaStream_t s = (cudaStream_t)stream;
    timing_begin("advect", s);
    advect_kernel<<<(unsigned)((n_sources + 255) / 256), 256, 0, s>>>(G, sources, n_sources, dt, out);
    timing_end("advect", s);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return failf(PIVBOS_ERR_CUDA, "advect: %s", cudaGetErrorString(e));
    return PIVBOS_OK;
}

pivbos_status pivbos_image_u16(const int64_t* image, int64_t n_pixels, double full_scale, uint16_t* out,
                               void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (n_pixels < 0) return failf(PIVBOS_ERR_INVALID_ARG, "n_pixels < 0");
    if (!(full_scale > 0.0) || !isfinite(full_scale)) return failf(PIVBOS_ERR_INVALID_ARG, "full_scale");
    if (n_pixels == 0) return PIVBOS_OK;
    if ((reinterpret_cast<uintptr_t>(image) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return failf(PIVBOS_ERR_INVALID_ARG, "image and out must be 16-byte aligned");
    int dev, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return failf(PIVBOS_ERR_CUDA, "cudaGetDevice");
    }
    pivbos_status st;
    if ((st = device_pointer(image, dev, "image")) || (st = device_pointer(out, dev, "out"))) return st;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (n_pixels / 8 + 255) / 256 + 1;
    const unsigned grid = (unsigned)std::min<int64_t>(need, (int64_t)(sms > 0 ? sms : 152) * 8);
    U16Scale S;
    S.d = std::max<long long>(1, llround(full_scale * 4294967296.0 / 65535.0));
    if (S.d > (1ll << 46)) return failf(PIVBOS_ERR_INVALID_ARG, "full_scale above 2^46 / 2^32 * 65535 rays");
    S.h = S.d / 2;
    S.thr = 65535ll * S.d - S.h;
    S.inv_d = (float)(1.0 / (double)S.d);
    cudaStream_t s = (cudaStream_t)stream;
    timing_begin("image_u16", s);
    image_u16_kernel<<<grid, 256, 0, s>>>(image, n_pixels, S, out);
    timing_end("image_u16", s);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return failf(PIVBOS_ERR_CUDA, "image_u16: %s", cudaGetErrorString(e));
    return PIVBOS_OK;
}

}  // extern "C"
