// The learned ray map (surrogate): host API of the MLP test hooks and of
// training / rendering with the surrogate.  The network maps a ray's entry
// state to the residual of its exit line (the paper has no learned part;
// this is a library facility built on the same tracer).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "handles.cuh"
#include "mlp.cuh"

namespace {

pivbos_status serr(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pivbos::set_last_error(buf);
    return st;
}

pivbos_status scuda(cudaError_t e, const char* what)
{
    return serr(e == cudaErrorMemoryAllocation ? PIVBOS_ERR_OOM : PIVBOS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

// Scoped device buffers for the test hooks.
struct HookBufs {
    pivbos::MlpDev d;
    pivbos::MlpWork w;
    float* x32 = nullptr;
    __nv_bfloat16* x = nullptr;
    float* t = nullptr;
    ~HookBufs()
    {
        pivbos::mlp_free(d);
        pivbos::mlp_work_free(w);
        cudaFree(x32);
        cudaFree(x);
        cudaFree(t);
    }
};

pivbos_status hook_setup(HookBufs& B, const float* params, const float* x, int32_t n, bool train)
{
    cudaError_t e = pivbos::mlp_alloc(B.d, 64);
    if (e == cudaSuccess && train) e = pivbos::mlp_work_alloc(B.w, n);
    if (e == cudaSuccess) e = cudaMalloc(&B.x32, sizeof(float) * (size_t)n * pivbos::kMlpIn);
    if (e == cudaSuccess) e = cudaMalloc(&B.x, sizeof(__nv_bfloat16) * (size_t)n * pivbos::kMlpIn);
    if (e == cudaSuccess)
        e = cudaMemcpy(B.d.params, params, sizeof(float) * pivbos::kMlpParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B.x32, x, sizeof(float) * (size_t)n * pivbos::kMlpIn, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return scuda(e, "mlp hook setup");
    const int64_t nx = (int64_t)n * pivbos::kMlpIn;
    f32_to_bf16_kernel<<<(unsigned)((nx + 255) / 256), 256>>>(B.x32, B.x, nx);
    e = pivbos::mlp_sync_bf16(B.d, 0);
    if (e != cudaSuccess) return scuda(e, "mlp weights to bf16");
    return PIVBOS_OK;
}

}  // namespace

extern "C" {

pivbos_status pivbos_mlp_forward(const float* params, const float* x, int32_t n, float* y)
{
    pivbos::set_last_error("");
    if (!params || !x || !y || n < 1) return serr(PIVBOS_ERR_INVALID_ARG, "mlp_forward arguments");
    HookBufs B;
    pivbos_status st = hook_setup(B, params, x, n, false);
    if (st) return st;
    float* dy = nullptr;
    cudaError_t e = cudaMalloc(&dy, sizeof(float) * (size_t)n * pivbos::kMlpOut);
    if (e == cudaSuccess) e = pivbos::mlp_forward(B.d, B.x, n, dy, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(float) * (size_t)n * pivbos::kMlpOut, cudaMemcpyDeviceToHost);
    cudaFree(dy);
    if (e != cudaSuccess) return scuda(e, "mlp_forward");
    return PIVBOS_OK;
}

pivbos_status pivbos_mlp_loss_grad(const float* params, const float* x, const float* t, int32_t n, float* grad,
                                   double* loss)
{
    pivbos::set_last_error("");
    if (!params || !x || !t || !grad || !loss || n < 1) return serr(PIVBOS_ERR_INVALID_ARG, "mlp_loss_grad arguments");
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
    if (e != cudaSuccess) return scuda(e, "mlp_loss_grad");
    *loss = lsum / ((double)n * pivbos::kMlpOut);
    return PIVBOS_OK;
}

}  // extern "C"
