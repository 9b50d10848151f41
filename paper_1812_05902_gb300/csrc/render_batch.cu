// Persistent batch render kernel (many frames in one launch).
#include "render_chunk.cuh"

namespace pivbos {

// Persistent batch kernel: CTAs pop work items (a frame and a chunk of its
// rays) from a device counter until the queue is empty.  Items are numbered
// frame by frame in the order the host chose (largest work first); the
// frame's parameters are copied to shared memory once per item.
template <int INTEG, bool CACHE, bool EXT>
__global__ void __launch_bounds__(kRenderThreads, CACHE ? 2 : kBatchMinBlocks)
batch_kernel(const BatchFrame* __restrict__ frames, const uint64_t* __restrict__ item_start, int n_frames,
             uint64_t total_items, unsigned long long* __restrict__ counter)
{
    __shared__ ChunkShared sh;
    __shared__ TraceParams sP;
    __shared__ unsigned long long s_item;
    __shared__ int s_frame;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long it = atomicAdd(counter, 1ull);
            s_item = it;
            int lo = 0, hi = n_frames - 1;
            if (it < total_items) {
                while (lo < hi) {   // last frame whose first item <= it
                    const int mid = (lo + hi + 1) >> 1;
                    if (item_start[mid] <= it) lo = mid; else hi = mid - 1;
                }
            }
            s_frame = lo;
        }
        __syncthreads();
        const unsigned long long it = s_item;
        if (it >= total_items) break;
        const int f = s_frame;
        {
            const int* src = reinterpret_cast<const int*>(&frames[f].p);
            int* dst = reinterpret_cast<int*>(&sP);
            for (int q = threadIdx.x; q < (int)(sizeof(TraceParams) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
        }
        __syncthreads();
        const BatchFrame& F = frames[f];
        const uint64_t first = (it - item_start[f]) * (uint64_t)F.rays_per_cta;
        const uint64_t last = min(first + F.rays_per_cta, F.total_rays);
        render_chunk<INTEG, CACHE, EXT>(sP, sh, first, last, F.image, F.stats);
    }
}

cudaError_t launch_batch(const BatchFrame* frames, const uint64_t* item_start, int n_frames, uint64_t total_items,
                         unsigned long long* counter, int integrator, bool cache, bool ext, int ctas_per_sm,
                         cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms * ctas_per_sm);
#define PV_BATCH(I, C, E) batch_kernel<I, C, E><<<grid, kRenderThreads, 0, s>>>(frames, item_start, n_frames, total_items, counter)
    PV_DISPATCH(integrator, cache, ext, PV_BATCH);
#undef PV_BATCH
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pivbos
