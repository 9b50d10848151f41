// The surrogate's MLP: 16 inputs -> 128 -> 128 -> 128 -> 128 -> 4, ReLU on the
// hidden layers, BF16 operands with FP32 accumulation on the tensor cores
// (tcgen05 for inference and training; the warp-level mma.sync kernels
// remain as the alternative PIVBOS_MLP_TC=0 selects), FP32 master weights
// and Adam.
//
// Parameter layout (FP32 master and gradients): layer by layer, W [out][in]
// row-major then b [out].  BF16 copies of the weights keep [out][in].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pivbos {

constexpr int kMlpIn = 16;      // padded input width
constexpr int kMlpHidden = 128;
constexpr int kMlpOut = 4;
constexpr int kMlpLayers = 5;
// (in, out) of each layer
__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? kMlpIn : kMlpHidden; }
__host__ __device__ constexpr int mlp_out(int l) { return l == kMlpLayers - 1 ? kMlpOut : kMlpHidden; }
__host__ __device__ constexpr int mlp_w_offset(int l)
{
    int off = 0;
    for (int q = 0; q < l; ++q) off += mlp_in(q) * mlp_out(q) + mlp_out(q);
    return off;
}
constexpr int kMlpParams = mlp_w_offset(kMlpLayers);           // 52,228
__host__ __device__ constexpr int mlp_wbf_offset(int l)
{
    int off = 0;
    for (int q = 0; q < l; ++q) off += mlp_in(q) * mlp_out(q);
    return off;
}
constexpr int kMlpWeights = mlp_wbf_offset(kMlpLayers);        // 51,712 BF16 weights

// Device buffers of one MLP (allocated by MlpState::create).
struct MlpDev {
    float* params = nullptr;       // FP32 master [kMlpParams]
    float* m = nullptr;            // Adam first moment
    float* v = nullptr;            // Adam second moment
    float* grad = nullptr;         // [kMlpParams]
    __nv_bfloat16* wbf = nullptr;  // BF16 weights [kMlpWeights]
    __nv_bfloat16* wbfT = nullptr; // the same, each layer transposed ([in][out]): the backward's operands
    float* partial = nullptr;      // dW/db partial sums [splits][max layer params]
    int splits = 0;
    int* status = nullptr;         // device word: nonzero after a tensor-core wait gave up
};

// Training workspace for batches of up to max_rows rows.
struct MlpWork {
    __nv_bfloat16* act = nullptr;  // hidden-layer outputs H1..H4 [4][rows][128]
    __nv_bfloat16* dz = nullptr;   // gradients: dZ of the hidden layers [4][rows][128], then dZ of the
                                   // output layer [rows][16] (the mma.sync path uses the first two planes)
    float* y = nullptr;            // outputs [rows][4]
    double* loss = nullptr;        // loss sum
    float* partial = nullptr;      // tcgen05 weight gradients per split [kMlpTcSplits][kMlpParams]
    int max_rows = 0;
};

constexpr int kMlpTcSplits = 32;   // row splits of the tcgen05 weight-gradient kernel

cudaError_t mlp_alloc(MlpDev& d, int splits);
void mlp_free(MlpDev& d);
cudaError_t mlp_work_alloc(MlpWork& w, int max_rows);
void mlp_work_free(MlpWork& w);

// BF16 copies of the master weights.
cudaError_t mlp_sync_bf16(const MlpDev& d, cudaStream_t s);
// Forward of n rows of X (BF16 [n][16]); Y [n][4] FP32.  With `work`
// (training) the hidden activations are kept and, given targets T
// ([n][4] FP32), the loss sum and dL/dY go to work.loss / work.dz[0].
cudaError_t mlp_forward(const MlpDev& d, const __nv_bfloat16* X, int n, float* Y, MlpWork* work, const float* T,
                        cudaStream_t s);
// Inference forward on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators), 128-row tiles.  Same inputs and outputs as mlp_forward
// without work; mlp_forward uses it for inference.
cudaError_t mlp_forward_tc(const MlpDev& d, const __nv_bfloat16* X, int n, float* Y, cudaStream_t s);
// PIVBOS_OK, or PIVBOS_ERR_DEVICE_TIMEOUT if a tensor-core wait gave up
// since the last call (synchronises with the device; clears the word).
int mlp_status(const MlpDev& d);
// Backward after a training forward: gradients of the mean loss into d.grad.
cudaError_t mlp_backward(MlpDev& d, const __nv_bfloat16* X, int n, MlpWork& work, cudaStream_t s);
// One Adam step (t counts from 1) on all parameters, then the BF16 copies.
cudaError_t mlp_adam(MlpDev& d, int t, float lr, cudaStream_t s);

// The surrogate's network kernel (the one its render launches) over n rows:
// R = B + MLP(X) * t_scale, X BF16 [n][16], B and R float4 [n] (device).
// Synchronous; *timed_out is set if a tensor-core wait gave up.
cudaError_t surr_net_apply(const MlpDev& net, const __nv_bfloat16* X, const float4* B, const float t_scale[4],
                           uint32_t n, float4* R, int* timed_out, cudaStream_t s);

}  // namespace pivbos
