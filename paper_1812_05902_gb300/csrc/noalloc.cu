// pivbos_render_noalloc: the render of pivbos_render for callers that must not
// allocate device memory.  Some callers cannot call cudaMalloc: a host
// application that has handed the whole device to its own memory pool and
// forbids allocations outside it, or a latency-critical loop in which the
// implicit device-wide synchronisation of cudaMalloc/cudaFree would stall
// other streams.  This entry point takes its only scratch (the Morton keys
// and the source permutation and sorted copy) from a file-scope device array
// of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "handles.cuh"

namespace {

constexpr size_t kStatusBytes = 256;
constexpr size_t kKeysBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * sizeof(uint64_t);
constexpr size_t kPermBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * sizeof(uint32_t);
constexpr size_t kSrcBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * 3 * sizeof(float2);
constexpr size_t kScratchBytes = kStatusBytes + kKeysBytes + kPermBytes + kSrcBytes;

}  // namespace

// [status word | sort keys (next power of two of n) | permutation (n) |
//  sources in Morton order as double-float (n x 3)]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char* g_scratch_addr[64] = {nullptr};

pivbos_status err(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pivbos::set_last_error(buf);
    return st;
}

// Device address of the scratch array on device `dev` (which must be
// current).  Looked up once per device: the host-side name of the array is
// not a device address.
pivbos_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 64) return err(PIVBOS_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return err(PIVBOS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return PIVBOS_OK;
}

pivbos::dfc split(double v)
{
    const float hi = (float)v;
    return pivbos::dfc{hi, (float)(v - (double)hi)};
}

pivbos_status device_buffer(const void* p, int dev, const char* what)
{
    if (!p) return err(PIVBOS_ERR_INVALID_ARG, "%s is NULL", what);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return err(PIVBOS_ERR_INVALID_ARG, "%s is not a CUDA pointer", what);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return err(PIVBOS_ERR_INVALID_ARG, "%s is not device memory", what);
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return err(PIVBOS_ERR_INVALID_ARG, "%s belongs to device %d, current is %d", what, a.device, dev);
    return PIVBOS_OK;
}

}  // namespace

extern "C" pivbos_status pivbos_render_noalloc(const pivbos_medium* m, const pivbos_optics* o,
                                               const double* sources, int64_t n_sources, int32_t rays_per_source,
                                               uint64_t seed, uint32_t frame, int integrator, double step,
                                               int64_t* image, int64_t* stats, void* stream)
{
    pivbos::set_last_error("");
    if (!o) return err(PIVBOS_ERR_INVALID_ARG, "optics handle is NULL");
    if (!image) return err(PIVBOS_ERR_INVALID_ARG, "image is NULL");
    if (n_sources < 0 || rays_per_source < 0) return err(PIVBOS_ERR_INVALID_ARG, "negative source or ray count");
    if (n_sources > PIVBOS_NOALLOC_MAX_SOURCES)
        return err(PIVBOS_ERR_UNSUPPORTED, "%lld sources exceed the %d that the fixed scratch array holds",
                   (long long)n_sources, (int)PIVBOS_NOALLOC_MAX_SOURCES);
    if (n_sources > 0 && !sources) return err(PIVBOS_ERR_INVALID_ARG, "sources is NULL");
    if (integrator != PIVBOS_EULER && integrator != PIVBOS_RK4)
        return err(PIVBOS_ERR_INVALID_ARG, "integrator %d", integrator);
    if (!(isfinite(step) && step > 0.0)) return err(PIVBOS_ERR_INVALID_ARG, "step must be finite and > 0");
    const uint64_t total = (uint64_t)n_sources * (uint64_t)rays_per_source;
    if (total > (1ull << 31)) return err(PIVBOS_ERR_OVERFLOW, "more than 2^31 rays in one render");

    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (o->device != dev) return err(PIVBOS_ERR_INVALID_ARG, "optics handle belongs to device %d", o->device);
    if (m && m->device != dev) return err(PIVBOS_ERR_INVALID_ARG, "medium handle belongs to device %d", m->device);
    pivbos_status st = device_buffer(image, dev, "image");
    if (st) return st;
    if (n_sources > 0) {
        st = device_buffer(sources, dev, "sources");
        if (st) return st;
    }
    if (stats) {
        st = device_buffer(stats, dev, "stats");
        if (st) return st;
    }
    unsigned char* scratch = nullptr;
    st = scratch_address(dev, &scratch);
    if (st) return st;
    if (total == 0) return PIVBOS_OK;

    pivbos::TraceParams p;
    memset(&p, 0, sizeof p);
    if (m) {
        p.m.present = 1;
        p.m.field = m->field;
        double diag2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            p.m.n[a] = m->n[a];
            p.m.h[a] = (float)m->spacing[a];
            p.m.inv_h[a] = (float)(1.0 / m->spacing[a]);
            p.m.inv_hd[a] = split(1.0 / m->spacing[a]);
            p.m.origin[a] = split(m->origin[a]);
            p.m.lo[a] = split(m->origin[a]);
            p.m.hi[a] = split(m->origin[a] + (double)(m->n[a] - 1) * m->spacing[a]);
            const double L = (double)(m->n[a] - 1) * m->spacing[a];
            diag2 += L * L;
        }
        const double ms = ceil(2.0 * sqrt(diag2) / step) + 4.0;
        if (ms > 2.0e9) return err(PIVBOS_ERR_UNSUPPORTED, "step too small for the box (%g steps)", ms);
        p.max_steps = (int)ms;
        p.m.z_key = (float)(m->origin[2] + 0.5 * (double)(m->n[2] - 1) * m->spacing[2]);
        pivbos::choose_gather(m, o, step, integrator, p);
    }
    p.o = o->d;
    p.sources = sources;
    p.n_sources = (uint32_t)n_sources;
    p.rays_per_source = (uint32_t)rays_per_source;
    p.seed = seed;
    p.frame = frame;
    p.step = (float)step;
    p.step_d = step;
    p.step_df = split(step);

    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)n_sources;
    uint32_t n_pow2 = 2;
    while (n_pow2 < n) n_pow2 <<= 1;
    int* status = (int*)scratch;
    uint64_t* keys = (uint64_t*)(scratch + kStatusBytes);
    uint32_t* perm = (uint32_t*)(scratch + kStatusBytes + kKeysBytes);
    float2* src_df = (float2*)(scratch + kStatusBytes + kKeysBytes + kPermBytes);
    // the array keeps the previous call's contents: the keys and the
    // permutation are fully rewritten below; the status word is cleared
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "status clear: %s", cudaGetErrorString(e));
    p.status_word = status;
    e = pivbos::launch_morton_sort(sources, n, keys, n_pow2, perm, src_df, s);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "sort: %s", cudaGetErrorString(e));
    p.perm = perm;
    p.src_df = src_df;
    e = pivbos::launch_render(p, integrator, image, stats, pivbos::rays_per_cta_setting(p), s);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    return PIVBOS_OK;
}
