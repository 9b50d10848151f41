/*
 * pivbos testing and measurement facilities -- libpivbos_testing.so.
 *
 * Not part of the product ABI (include/pivbos.h): these calls exist so that
 * tests can check the product library's kernels element by element against
 * an FP64 reference, and so that benchmarks can measure a roofline
 * denominator.  None has a counterpart in the paper.  The library links
 * libpivbos.so and runs its kernels; it shares pivbos_last_error() with it.
 * Every call but pivbos_plan_bins (host only) runs on the current device,
 * synchronously, and allocates its own device memory.  Errors: INVALID_ARG (NULL pointers, n < 1), OOM, CUDA,
 * DEVICE_TIMEOUT (a bounded tensor-core wait gave up).
 */
#ifndef PIVBOS_TESTING_H
#define PIVBOS_TESTING_H

#include <stdint.h>

#include "pivbos.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The surrogate's network, 16 inputs -> 128 -> 128 -> 128 -> 128 -> 4, ReLU
 * on the hidden layers, BF16 operands and FP32 accumulation.  params: host
 * float [PIVBOS_MLP_PARAMS], layer by layer W [out][in] then b [out]; the
 * calls round weights and inputs to BF16 as the product path does.  x: host
 * float [n][16]; inputs 14 and 15 must be zero (the inference kernels carry
 * the first layer's bias through them).
 *
 * pivbos_mlp_forward: the inference forward (tensor cores, tcgen05), y: host
 * float [n][4].
 * pivbos_mlp_train_forward: the training forward (the kernel training uses),
 * y: host float [n][4].
 * pivbos_mlp_loss_grad: the training forward and backward of the mean
 * squared error over n x 4 outputs against t (host float [n][4]); grad: host
 * float [PIVBOS_MLP_PARAMS], loss: the mean. */
pivbos_status pivbos_mlp_forward(const float* params, const float* x, int32_t n, float* y);
pivbos_status pivbos_mlp_train_forward(const float* params, const float* x, int32_t n, float* y);
pivbos_status pivbos_mlp_loss_grad(const float* params, const float* x, const float* t, int32_t n,
                                   float* grad, double* loss);

/* n_steps Adam steps of the training kernel (beta1 0.9, beta2 0.999, eps
 * 1e-8, bias-corrected, step numbers t0, t0 + 1, ...): params, m, v (host
 * float [PIVBOS_MLP_PARAMS], updated in place) with the gradients grads
 * (host float [n_steps][PIVBOS_MLP_PARAMS]) and learning rates lr (host
 * float [n_steps]).  wbf (host uint16 [51712], may be NULL) receives the BF16
 * weight copy the kernel writes (bias entries excluded), as raw bits. */
pivbos_status pivbos_mlp_adam_steps(float* params, float* m, float* v, const float* grads, int32_t n_steps,
                                    int32_t t0, const float* lr, uint16_t* wbf);

/* The surrogate render's network kernel over n rows, as the render runs it:
 * r[i] = b[i] + MLP(x[i]) * t_scale, with x host float [n][16] (rounded to
 * BF16), b and r host float [n][4], t_scale host float [4].  The kernel
 * carries every bias through the tensor core as a BF16 leading part plus a
 * BF16 remainder. */
pivbos_status pivbos_surrogate_net_apply(const float* params, const float* x, const float* b,
                                         const float t_scale[4], int32_t n, float* r);

/* The bandwidth of the current device's L1 data path for coalesced 16-byte
 * loads from an L1-resident buffer (every SM streams 48 KB), in bytes per
 * second -- the denominator of the field-gather rooflines. */
pivbos_status pivbos_probe_l1_bandwidth(double* bytes_per_second);

/* The surrogate's per-bin plan, as pivbos_surrogate_train makes it (host
 * code, no device): for each of n_bins entry bins (a multiple of 32) with
 * counts[b] held-out rays, their summed squared sensor errors err2p[b]
 * (projection alone) and err2n[b] (with the network's correction) and their
 * plain-path steps steps[b], serve the bin by the projection alone, the
 * projection with the correction (only if with_net) or the plain fallback,
 * at the least render cost (in plain steps; segments projection segments)
 * whose served squared error stays within budget2; bins with fewer than
 * min_count rays fall back.  served, network: n_bins / 32 words of bits
 * (host, written).  out (host double [5]): served squared error, served
 * steps, served rays, network rays, cost.  The paper has no counterpart: the
 * learned surrogate is an addition to the method. */
pivbos_status pivbos_plan_bins(const double* err2n, const double* err2p, const double* steps,
                               const uint32_t* counts, int32_t n_bins, int32_t min_count, double budget2,
                               int32_t segments, int32_t with_net, uint32_t* served, uint32_t* network,
                               double* out);

#ifdef __cplusplus
}
#endif

#endif /* PIVBOS_TESTING_H */
