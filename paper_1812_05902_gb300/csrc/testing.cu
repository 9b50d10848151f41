// libpivbos_testing.so: measurement and checking facilities kept out of the
// product library (include/pivbos_testing.h).  The network hooks run the
// product library's own kernels (linked from libpivbos.so) on host buffers,
// so tests can compare them element by element with an FP64 reference; the
// L1 probe measures the denominator of the field-gather rooflines.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "handles.cuh"
#include "mlp.cuh"
#include "../../include/pivbos_testing.h"

namespace {

pivbos_status terr(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pivbos::set_last_error(buf);
    return st;
}

pivbos_status tcuda(cudaError_t e, const char* what)
{
    return terr(e == cudaErrorMemoryAllocation ? PIVBOS_ERR_OOM : PIVBOS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

// Scoped device buffers of one hook call.
struct HookBufs {
    pivbos::MlpDev d;
    pivbos::MlpWork w;
    float* x32 = nullptr;
    __nv_bfloat16* x = nullptr;
    float* t = nullptr;
    float4* b = nullptr;
    float4* r = nullptr;
    ~HookBufs()
    {
        pivbos::mlp_free(d);
        pivbos::mlp_work_free(w);
        cudaFree(x32);
        cudaFree(x);
        cudaFree(t);
        cudaFree(b);
        cudaFree(r);
    }
};

// Network parameters and (if n > 0) inputs on the device; BF16 copies of both.
pivbos_status hook_setup(HookBufs& B, const float* params, const float* x, int32_t n, bool train)
{
    cudaError_t e = pivbos::mlp_alloc(B.d, 64);
    if (e == cudaSuccess && train) e = pivbos::mlp_work_alloc(B.w, n);
    if (e == cudaSuccess)
        e = cudaMemcpy(B.d.params, params, sizeof(float) * pivbos::kMlpParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n > 0) {
        e = cudaMalloc(&B.x32, sizeof(float) * (size_t)n * pivbos::kMlpIn);
        if (e == cudaSuccess) e = cudaMalloc(&B.x, sizeof(__nv_bfloat16) * (size_t)n * pivbos::kMlpIn);
        if (e == cudaSuccess)
            e = cudaMemcpy(B.x32, x, sizeof(float) * (size_t)n * pivbos::kMlpIn, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            const int64_t nx = (int64_t)n * pivbos::kMlpIn;
            f32_to_bf16_kernel<<<(unsigned)((nx + 255) / 256), 256>>>(B.x32, B.x, nx);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = pivbos::mlp_sync_bf16(B.d, 0);
    if (e != cudaSuccess) return tcuda(e, "mlp hook setup");
    return PIVBOS_OK;
}

}  // namespace

extern "C" {

pivbos_status pivbos_mlp_forward(const float* params, const float* x, int32_t n, float* y)
{
    pivbos::set_last_error("");
    if (!params || !x || !y || n < 1) return terr(PIVBOS_ERR_INVALID_ARG, "mlp_forward arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, x, n, false);
    if (st) return st;
    float* dy = nullptr;
    cudaError_t e = cudaMalloc(&dy, sizeof(float) * (size_t)n * pivbos::kMlpOut);
    if (e == cudaSuccess) e = pivbos::mlp_forward(B.d, B.x, n, dy, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(float) * (size_t)n * pivbos::kMlpOut, cudaMemcpyDeviceToHost);
    cudaFree(dy);
    if (e != cudaSuccess) return tcuda(e, "mlp_forward");
    if (pivbos::mlp_status(B.d)) return terr(PIVBOS_ERR_DEVICE_TIMEOUT, "mlp_forward: a tensor-core wait gave up");
    return PIVBOS_OK;
}

pivbos_status pivbos_mlp_train_forward(const float* params, const float* x, int32_t n, float* y)
{
    pivbos::set_last_error("");
    if (!params || !x || !y || n < 1) return terr(PIVBOS_ERR_INVALID_ARG, "mlp_train_forward arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, x, n, true);
    if (st) return st;
    cudaError_t e = pivbos::mlp_forward(B.d, B.x, n, B.w.y, &B.w, nullptr, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, B.w.y, sizeof(float) * (size_t)n * pivbos::kMlpOut, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "mlp_train_forward");
    if (pivbos::mlp_status(B.d)) return terr(PIVBOS_ERR_DEVICE_TIMEOUT, "mlp_train_forward: a wait gave up");
    return PIVBOS_OK;
}

pivbos_status pivbos_mlp_loss_grad(const float* params, const float* x, const float* t, int32_t n, float* grad,
                                   double* loss)
{
    pivbos::set_last_error("");
    if (!params || !x || !t || !grad || !loss || n < 1) return terr(PIVBOS_ERR_INVALID_ARG, "mlp_loss_grad arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, x, n, true);
    if (st) return st;
    cudaError_t e = cudaMalloc(&B.t, sizeof(float) * (size_t)n * pivbos::kMlpOut);
    if (e == cudaSuccess) e = cudaMemcpy(B.t, t, sizeof(float) * (size_t)n * pivbos::kMlpOut, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = pivbos::mlp_forward(B.d, B.x, n, B.w.y, &B.w, B.t, 0);
    if (e == cudaSuccess) e = pivbos::mlp_backward(B.d, B.x, n, B.w, 0);
    if (e == cudaSuccess) e = cudaMemcpy(grad, B.d.grad, sizeof(float) * pivbos::kMlpParams, cudaMemcpyDeviceToHost);
    double lsum = 0.0;
    if (e == cudaSuccess) e = cudaMemcpy(&lsum, B.w.loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "mlp_loss_grad");
    if (pivbos::mlp_status(B.d)) return terr(PIVBOS_ERR_DEVICE_TIMEOUT, "mlp_loss_grad: a wait gave up");
    *loss = lsum / ((double)n * pivbos::kMlpOut);
    return PIVBOS_OK;
}

pivbos_status pivbos_mlp_adam_steps(float* params, float* m, float* v, const float* grads, int32_t n_steps,
                                    int32_t t0, const float* lr, uint16_t* wbf)
{
    pivbos::set_last_error("");
    if (!params || !m || !v || !grads || !lr || n_steps < 1 || t0 < 1)
        return terr(PIVBOS_ERR_INVALID_ARG, "mlp_adam_steps arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, nullptr, 0, false);
    if (st) return st;
    const size_t bytes = sizeof(float) * pivbos::kMlpParams;
    cudaError_t e = cudaMemcpy(B.d.m, m, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B.d.v, v, bytes, cudaMemcpyHostToDevice);
    for (int q = 0; q < n_steps && e == cudaSuccess; ++q) {
        e = cudaMemcpy(B.d.grad, grads + (size_t)q * pivbos::kMlpParams, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = pivbos::mlp_adam(B.d, t0 + q, lr[q], 0);
    }
    if (e == cudaSuccess) e = cudaMemcpy(params, B.d.params, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(m, B.d.m, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(v, B.d.v, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && wbf)
        e = cudaMemcpy(wbf, B.d.wbf, sizeof(uint16_t) * pivbos::kMlpWeights, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "mlp_adam_steps");
    return PIVBOS_OK;
}

pivbos_status pivbos_surrogate_net_apply(const float* params, const float* x, const float* b, const float t_scale[4],
                                         int32_t n, float* r)
{
    pivbos::set_last_error("");
    if (!params || !x || !b || !t_scale || !r || n < 1) return terr(PIVBOS_ERR_INVALID_ARG, "net_apply arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, x, n, false);
    if (st) return st;
    cudaError_t e = cudaMalloc(&B.b, sizeof(float4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&B.r, sizeof(float4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(B.b, b, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice);
    int timed_out = 0;
    if (e == cudaSuccess) e = pivbos::surr_net_apply(B.d, B.x, B.b, t_scale, (uint32_t)n, B.r, &timed_out, 0);
    if (e == cudaSuccess) e = cudaMemcpy(r, B.r, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "surrogate_net_apply");
    if (timed_out) return terr(PIVBOS_ERR_DEVICE_TIMEOUT, "surrogate_net_apply: a tensor-core wait gave up");
    return PIVBOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The L1 data path's bandwidth for 16-byte loads.  Every CTA streams one
// 48 KB buffer (L1-resident after the first pass) with coalesced float4
// loads.
// ---------------------------------------------------------------------------
namespace {

constexpr int kProbeFloat4 = 3072;   // 48 KB

__global__ void __launch_bounds__(256) l1_probe_kernel(const float4* __restrict__ buf, int iters,
                                                       float* __restrict__ sink)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int q = threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        const float4 v = __ldg(buf + q);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
        q += 256;
        if (q >= kProbeFloat4) q -= kProbeFloat4;
    }
    // keeps the loads; the buffer holds zeros, so nothing is written
    if (acc.x + acc.y + acc.z + acc.w != 0.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc.x;
}

}  // namespace

extern "C" pivbos_status pivbos_probe_l1_bandwidth(double* bytes_per_second)
{
    pivbos::set_last_error("");
    if (!bytes_per_second) return terr(PIVBOS_ERR_INVALID_ARG, "bytes_per_second is NULL");
    int dev, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return terr(PIVBOS_ERR_CUDA, "cudaGetDevice");
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (sms > 0 ? sms : 152) * 8, iters = 4096;
    float4* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, kProbeFloat4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void**)&sink, (size_t)blocks * 256 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, kProbeFloat4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0.f;
    if (e == cudaSuccess) {
        l1_probe_kernel<<<blocks, 256>>>(buf, iters, sink);   // warm-up
        cudaEventRecord(a);
        for (int r = 0; r < 5; ++r) l1_probe_kernel<<<blocks, 256>>>(buf, iters, sink);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return tcuda(e, "L1 probe");
    *bytes_per_second = 5.0 * (double)blocks * 256.0 * (double)iters * 16.0 / (ms * 1e-3);
    return PIVBOS_OK;
}

namespace pivbos {
// The surrogate's per-bin plan (surrogate.cu, exported by libpivbos.so; host
// code): for each entry bin the projection alone, with the network's
// correction, or the plain fallback, the least render cost under the
// squared-error budget budget2.  ok and net: n_bins / 32 words of bits.
// Returns the plan's cost in plain steps.
double plan_bins(const double* err2n, const double* err2p, const double* steps, const unsigned* cnt, int n_bins,
                 int min_count, double budget2, int segments, bool with_net, uint32_t* ok, uint32_t* net,
                 double* err2_out, double* rays_out, double* net_rays_out);
}  // namespace pivbos

extern "C" pivbos_status pivbos_plan_bins(const double* err2n, const double* err2p, const double* steps,
                                          const uint32_t* counts, int32_t n_bins, int32_t min_count, double budget2,
                                          int32_t segments, int32_t with_net, uint32_t* served, uint32_t* network,
                                          double* out)
{
    pivbos::set_last_error("");
    if (!err2n || !err2p || !steps || !counts || !served || !network || !out)
        return terr(PIVBOS_ERR_INVALID_ARG, "NULL argument");
    if (n_bins < 32 || n_bins % 32 != 0) return terr(PIVBOS_ERR_INVALID_ARG, "n_bins must be a positive multiple of 32");
    if (segments < 1 || !(budget2 >= 0.0)) return terr(PIVBOS_ERR_INVALID_ARG, "segments < 1 or budget2 < 0");
    out[4] = pivbos::plan_bins(err2n, err2p, steps, counts, n_bins, min_count, budget2, segments, with_net != 0, served,
                               network, &out[0], &out[2], &out[3]);
    // the plan's plain steps saved: the served bins' steps
    double saved = 0.0;
    for (int b = 0; b < n_bins; ++b)
        if ((served[b >> 5] >> (b & 31)) & 1u) saved += steps[b];
    out[1] = saved;
    return PIVBOS_OK;
}

