// Render kernels: the fused per-ray path (Sec. 3.1-3.4) with the deposit into
// a shared-memory tile, the per-ray exit-state kernel used for parity, and
// the fixed-point -> float finalisation.
#include "render_chunk.cuh"

namespace pivbos {

template <int INTEG, bool CACHE, bool EXT>
__global__ void __launch_bounds__(kRenderThreads, CACHE ? 3 : kRenderMinBlocks)
render_kernel(const TraceParams P, int64_t* __restrict__ image, int64_t* __restrict__ stats,
              uint32_t rays_per_cta, uint64_t total_rays)
{
    __shared__ ChunkShared sh;
    const uint64_t first = (uint64_t)blockIdx.x * rays_per_cta;
    const uint64_t last = min(first + rays_per_cta, total_rays);
    render_chunk<INTEG, CACHE, EXT>(P, sh, first, last, image, stats);
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
        st.opl = 0.0;
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
    const bool ext = optics_ext(p.o);
#define PV_RENDER(I, C, E) render_kernel<I, C, E><<<(unsigned)blocks, kRenderThreads, 0, s>>>(p, image, stats, rays_per_cta, total)
    PV_DISPATCH(integrator, cache, ext, PV_RENDER);
#undef PV_RENDER
    timing_end("render", s);
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
