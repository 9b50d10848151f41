// Self-test of the failure detection (no counterpart in the paper): the
// bounded mbarrier wait of the tensor-core kernels, on a barrier nothing
// arrives at, gives up and reports a device timeout instead of hanging.
#include "handles.cuh"
#include "umma.cuh"

namespace pivbos {

__global__ void wait_timeout_kernel(uint32_t polls, int* __restrict__ status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) umma::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !umma::mbar_wait(&bar, 0u, polls))
        atomicCAS(status, 0, (int)PIVBOS_ERR_DEVICE_TIMEOUT);
}

}  // namespace pivbos

extern "C" pivbos_status pivbos_selftest_wait_timeout(uint32_t polls, void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (polls == 0 || polls > (1u << 20)) return failf(PIVBOS_ERR_INVALID_ARG, "polls outside [1, 2^20]");
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return failf(PIVBOS_ERR_CUDA, "cudaGetDevice");
    }
    int* sw = nullptr;
    pivbos_status st = device_status_word(dev, &sw);
    if (st) return st;
    wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(polls, sw);
    count_launches(1);
    return cuda_status(cudaGetLastError(), "self-test launch");
}
