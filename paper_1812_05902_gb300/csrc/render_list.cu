// Persistent render kernel over a device-side list of rays (the surrogate's
// fallback rays).
#include "render_chunk.cuh"

namespace pivbos {

// Persistent kernel over a device-side ray list (the surrogate's fallback
// rays): chunks of rays_per_cta consecutive list entries.
template <int INTEG, bool CACHE, bool EXT>
__global__ void __launch_bounds__(kRenderThreads, CACHE ? 2 : kRenderMinBlocks)
list_kernel(const TraceParams P, const unsigned long long* __restrict__ count, uint32_t capacity,
            int64_t* __restrict__ image, int64_t* __restrict__ stats, uint32_t rays_per_cta,
            unsigned long long* __restrict__ counter)
{
    __shared__ ChunkShared sh;
    __shared__ unsigned long long s_item;
    const uint64_t n = min(*count, (unsigned long long)capacity);
    const uint64_t items = (n + rays_per_cta - 1) / rays_per_cta;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ull);
        __syncthreads();
        const uint64_t it = s_item;
        if (it >= items) break;
        const uint64_t first = it * rays_per_cta;
        render_chunk<INTEG, CACHE, EXT>(P, sh, first, min(first + rays_per_cta, n), image, stats);
    }
}

cudaError_t launch_list(const TraceParams& p, int integrator, const unsigned long long* count, uint32_t capacity,
                        int64_t* image, int64_t* stats, uint32_t rays_per_cta, unsigned long long* counter,
                        cudaStream_t s)
{
    if (rays_per_cta == 0 || rays_per_cta > (uint32_t)kMaxOrderRays) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool cache = p.cell_cache != 0;
    const unsigned grid = (unsigned)(sms * (cache ? 2 : kRenderMinBlocks));
    const bool ext = optics_ext(p.o);
#define PV_LIST(I, C, E) list_kernel<I, C, E><<<grid, kRenderThreads, 0, s>>>(p, count, capacity, image, stats, rays_per_cta, counter)
    PV_DISPATCH(integrator, cache, ext, PV_LIST);
#undef PV_LIST
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pivbos
