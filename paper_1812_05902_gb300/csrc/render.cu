// Render kernels: the fused per-ray path (Sec. 3.1-3.4) with the deposit into
// a shared-memory tile, the per-ray exit-state kernel used for parity, and
// the fixed-point -> float finalisation.
#include "trace.cuh"

namespace pivbos {

constexpr int kRenderThreads = 256;
constexpr int kRenderMinBlocks = 4;   // CTAs per SM the register budget must allow
constexpr int kBatchMinBlocks = 3;    // ... for the persistent batch kernel (4 would spill 112 B)
// Work: the flattened (Morton slot, ray) index space (sources in Morton order,
// read as double-float from P.src_df) is cut into chunks of
// rays_per_cta consecutive rays; a CTA takes one chunk, so its rays come
// from one source or a few neighbouring ones and their spots fall in one
// 32x32 shared tile anchored at the first hit.
// Shared memory of one CTA working on one chunk of rays.
struct ChunkShared {
    unsigned long long tile[kTileW * kTileH];
    uint32_t order[kMaxOrderRays];
    unsigned long long cnt[PIVBOS_RAY_NSTATUS];
    int anchor_tid, ax, ay;
};

// Rays [first, last) of the flattened (Morton slot, ray) space of one render:
// trace (in mid-plane Morton order in dense media), deposit into the shared
// tile anchored at the first hit, flush the tile, add the status counts.
// Every thread of the CTA must call it; it leaves `sh` free for reuse.
template <int INTEG, bool CACHE>
__device__ __forceinline__ void render_chunk(const TraceParams& P, ChunkShared& sh, uint64_t first, uint64_t last,
                                             int64_t* __restrict__ image, int64_t* __restrict__ stats)
{
    for (int q = threadIdx.x; q < kTileW * kTileH; q += blockDim.x) sh.tile[q] = 0ull;
    if (threadIdx.x == 0) {
        sh.anchor_tid = 0x7fffffff;
        sh.ax = -(1 << 28);
        sh.ay = -(1 << 28);
    }
    if (threadIdx.x < PIVBOS_RAY_NSTATUS) sh.cnt[threadIdx.x] = 0ull;
    __syncthreads();

    const uint32_t rps = P.rays_per_source;
    unsigned cnt[PIVBOS_RAY_NSTATUS] = {0, 0, 0, 0, 0, 0};

    // In a dense medium, trace the CTA's rays in the order of where they
    // cross the box: a warp then gathers from a few neighbouring cells
    // instead of the whole cone of a source.
    const uint32_t n_here = (uint32_t)(last - first);
    const bool reorder = P.reorder && n_here <= (uint32_t)kMaxOrderRays;
    if (reorder) order_chunk(P, sh.order, first, n_here);
    // one uniform loop over the chunk's rays; after the first round every
    // thread's first hit is known and the lowest-thread hit anchors the tile
    const int rounds = (int)((n_here + blockDim.x - 1) / blockDim.x);
    int ax = -(1 << 28), ay = -(1 << 28);
    for (int round = 0; round < rounds; ++round) {
        const uint32_t e = (uint32_t)round * blockDim.x + threadIdx.x;
        const bool active = e < n_here;
        const uint64_t idx = first + (reorder && active ? (sh.order[e] & 0x7ffu) : e);
        RayOut r;
        r.status = PIVBOS_RAY_MISS;
        if (active) {
            const uint32_t flat = P.ray_list ? __ldg(P.ray_list + idx) : (uint32_t)idx;
            const uint32_t slot = flat / rps, k = flat - slot * rps;
            const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
            const float2* s = P.src_df + 3 * (size_t)slot;
            const float2 a = __ldg(s), b = __ldg(s + 1), c = __ldg(s + 2);
            trace_ray<INTEG, CACHE>(P, df{a.x, a.y}, df{b.x, b.y}, df{c.x, c.y}, sid, k, r, nullptr);
            cnt[r.status]++;
        }
        if (round == 0) {
            if (active && r.status == PIVBOS_RAY_REACHED) atomicMin(&sh.anchor_tid, (int)threadIdx.x);
            __syncthreads();
            if ((int)threadIdx.x == sh.anchor_tid) {
                float f;
                sh.ax = df_floor(r.px, f) - kTileW / 2;
                sh.ay = df_floor(r.py, f) - kTileH / 2;
            }
            __syncthreads();
            ax = sh.ax;
            ay = sh.ay;
        }
        if (active && r.status == PIVBOS_RAY_REACHED) deposit_ray(P.o, r.px, r.py, sh.tile, ax, ay, image);
    }
    if (stats) {
#pragma unroll
        for (int q = 0; q < PIVBOS_RAY_NSTATUS; ++q) {
            unsigned v = cnt[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sh.cnt[q], (unsigned long long)v);
        }
    }
    __syncthreads();
    // flush the tile: one global atomic per touched pixel
    for (int q = threadIdx.x; q < kTileW * kTileH; q += blockDim.x) {
        const unsigned long long v = sh.tile[q];
        if (v) {
            const int gx = ax + (q % kTileW), gy = ay + (q / kTileW);
            atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * P.o.W + gx]), v);
        }
    }
    if (stats && threadIdx.x < PIVBOS_RAY_NSTATUS && sh.cnt[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[threadIdx.x]), sh.cnt[threadIdx.x]);
    __syncthreads();
}

template <int INTEG, bool CACHE>
__global__ void __launch_bounds__(kRenderThreads, CACHE ? 2 : kRenderMinBlocks)
render_kernel(const TraceParams P, int64_t* __restrict__ image, int64_t* __restrict__ stats,
              uint32_t rays_per_cta, uint64_t total_rays)
{
    __shared__ ChunkShared sh;
    const uint64_t first = (uint64_t)blockIdx.x * rays_per_cta;
    const uint64_t last = min(first + rays_per_cta, total_rays);
    render_chunk<INTEG, CACHE>(P, sh, first, last, image, stats);
}

// Persistent batch kernel: CTAs pop work items (a frame and a chunk of its
// rays) from a device counter until the queue is empty.  Items are numbered
// frame by frame in the order the host chose (largest work first); the
// frame's parameters are copied to shared memory once per item.
template <int INTEG, bool CACHE>
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
        render_chunk<INTEG, CACHE>(sP, sh, first, last, F.image, F.stats);
    }
}

// Persistent kernel over a device-side ray list (the surrogate's fallback
// rays): chunks of rays_per_cta consecutive list entries.
template <int INTEG, bool CACHE>
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
        render_chunk<INTEG, CACHE>(P, sh, first, min(first + rays_per_cta, n), image, stats);
    }
}

template <int INTEG>
__global__ void __launch_bounds__(128)
trace_states_kernel(const TraceParams P, const int64_t* __restrict__ ray_ids, int64_t n,
                    pivbos_ray_state* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t id = ray_ids ? ray_ids[q] : q;
    const uint32_t rps = P.rays_per_source;
    pivbos_ray_state st;
    RayOut r;
    if (id < 0 || id >= (int64_t)P.n_sources * rps) {
        // an id outside the render: reported as a miss with no geometry
        for (int a = 0; a < 3; ++a) { st.vol_pos[a] = 0.0; st.vol_dir[a] = 0.0; st.sensor_dir[a] = 0.0; }
        st.sensor_xy[0] = st.sensor_xy[1] = 0.0;
        st.status = PIVBOS_RAY_MISS;
        st.steps = 0;
        atomicCAS(P.status_word, 0, (int)PIVBOS_ERR_INVALID_ARG);
    } else {
        const uint32_t sid = (uint32_t)(id / rps), k = (uint32_t)(id - (int64_t)sid * rps);
        const double* s = P.sources + 3 * (size_t)sid;
        trace_ray<INTEG, false>(P, df_from_double(s[0]), df_from_double(s[1]), df_from_double(s[2]),
                                sid + P.source_offset, k, r, &st);
    }
    out[q] = st;
}

__global__ void finalize_kernel(const int64_t* __restrict__ img, int64_t n, float* __restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
        out[q] = (float)((double)img[q] * 0x1p-32);
}

cudaError_t launch_render(const TraceParams& p, int integrator, int64_t* image, int64_t* stats,
                          uint32_t rays_per_cta, cudaStream_t s)
{
    const uint64_t total = (uint64_t)p.n_sources * p.rays_per_source;
    if (total == 0) return cudaSuccess;
    const uint64_t blocks = (total + rays_per_cta - 1) / rays_per_cta;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    timing_begin("render", s);
    const bool cache = p.cell_cache != 0;
    if (integrator == PIVBOS_RK4) {
        if (cache)
            render_kernel<PIVBOS_RK4, true><<<(unsigned)blocks, kRenderThreads, 0, s>>>(p, image, stats, rays_per_cta, total);
        else
            render_kernel<PIVBOS_RK4, false><<<(unsigned)blocks, kRenderThreads, 0, s>>>(p, image, stats, rays_per_cta, total);
    } else {
        if (cache)
            render_kernel<PIVBOS_EULER, true><<<(unsigned)blocks, kRenderThreads, 0, s>>>(p, image, stats, rays_per_cta, total);
        else
            render_kernel<PIVBOS_EULER, false><<<(unsigned)blocks, kRenderThreads, 0, s>>>(p, image, stats, rays_per_cta, total);
    }
    timing_end("render", s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchFrame* frames, const uint64_t* item_start, int n_frames, uint64_t total_items,
                         unsigned long long* counter, int integrator, bool cache, int ctas_per_sm, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms * ctas_per_sm);
    if (integrator == PIVBOS_RK4) {
        if (cache)
            batch_kernel<PIVBOS_RK4, true><<<grid, kRenderThreads, 0, s>>>(frames, item_start, n_frames, total_items, counter);
        else
            batch_kernel<PIVBOS_RK4, false><<<grid, kRenderThreads, 0, s>>>(frames, item_start, n_frames, total_items, counter);
    } else {
        if (cache)
            batch_kernel<PIVBOS_EULER, true><<<grid, kRenderThreads, 0, s>>>(frames, item_start, n_frames, total_items, counter);
        else
            batch_kernel<PIVBOS_EULER, false><<<grid, kRenderThreads, 0, s>>>(frames, item_start, n_frames, total_items, counter);
    }
    count_launches(1);
    return cudaGetLastError();
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
    if (integrator == PIVBOS_RK4) {
        if (cache)
            list_kernel<PIVBOS_RK4, true><<<grid, kRenderThreads, 0, s>>>(p, count, capacity, image, stats, rays_per_cta, counter);
        else
            list_kernel<PIVBOS_RK4, false><<<grid, kRenderThreads, 0, s>>>(p, count, capacity, image, stats, rays_per_cta, counter);
    } else {
        if (cache)
            list_kernel<PIVBOS_EULER, true><<<grid, kRenderThreads, 0, s>>>(p, count, capacity, image, stats, rays_per_cta, counter);
        else
            list_kernel<PIVBOS_EULER, false><<<grid, kRenderThreads, 0, s>>>(p, count, capacity, image, stats, rays_per_cta, counter);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trace_states(const TraceParams& p, int integrator, const int64_t* ray_ids,
                                int64_t n_rays, pivbos_ray_state* out, cudaStream_t s)
{
    if (n_rays == 0) return cudaSuccess;
    const int64_t blocks = (n_rays + 127) / 128;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    timing_begin("trace_states", s);
    if (integrator == PIVBOS_RK4)
        trace_states_kernel<PIVBOS_RK4><<<(unsigned)blocks, 128, 0, s>>>(p, ray_ids, n_rays, out);
    else
        trace_states_kernel<PIVBOS_EULER><<<(unsigned)blocks, 128, 0, s>>>(p, ray_ids, n_rays, out);
    timing_end("trace_states", s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const int64_t* image, int64_t n, float* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    timing_begin("finalize", s);
    finalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(image, n, out);
    timing_end("finalize", s);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pivbos
