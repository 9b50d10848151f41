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

constexpr size_t kHeadBytes = 256;    // reserved (alignment of what follows)
constexpr size_t kKeysBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * sizeof(uint64_t);
constexpr size_t kPermBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * sizeof(uint32_t);
constexpr size_t kSrcBytes = (size_t)PIVBOS_NOALLOC_MAX_SOURCES * 3 * sizeof(float2);
constexpr size_t kScratchBytes = kHeadBytes + kKeysBytes + kPermBytes + kSrcBytes;

}  // namespace

// [reserved | sort keys (next power of two of n) | permutation (n) |
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
    if (!image) return err(PIVBOS_ERR_INVALID_ARG, "image is NULL");
    if (n_sources > PIVBOS_NOALLOC_MAX_SOURCES)
        return err(PIVBOS_ERR_UNSUPPORTED, "%lld sources exceed the %d that the fixed scratch array holds",
                   (long long)n_sources, (int)PIVBOS_NOALLOC_MAX_SOURCES);
    // the same checks and kernel parameters as pivbos_render (no allocation:
    // the device status word is a fixed device array too)
    pivbos::TraceParams p;
    int dev = 0;
    uint64_t total = 0;
    pivbos_status st = pivbos::prepare_trace(m, o, sources, n_sources, 1, rays_per_source, seed, frame, integrator,
                                             step, &p, &dev, &total);
    if (st) return st;
    st = device_buffer(image, dev, "image");
    if (st) return st;
    if (stats) {
        st = device_buffer(stats, dev, "stats");
        if (st) return st;
    }
    unsigned char* scratch = nullptr;
    st = scratch_address(dev, &scratch);
    if (st) return st;
    if (total == 0) return PIVBOS_OK;

    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)n_sources;
    uint32_t n_pow2 = 2;
    while (n_pow2 < n) n_pow2 <<= 1;
    // the array keeps the previous call's contents: the keys, the permutation
    // and the sorted sources are fully rewritten by the sort before the
    // render reads them
    uint64_t* keys = (uint64_t*)(scratch + kHeadBytes);
    uint32_t* perm = (uint32_t*)(scratch + kHeadBytes + kKeysBytes);
    float2* src_df = (float2*)(scratch + kHeadBytes + kKeysBytes + kPermBytes);
    cudaError_t e = pivbos::launch_morton_sort(sources, n, keys, n_pow2, perm, src_df, s);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "sort: %s", cudaGetErrorString(e));
    p.perm = perm;
    p.src_df = src_df;
    e = pivbos::launch_render(p, integrator, image, stats, pivbos::rays_per_cta_setting(p), s);
    if (e != cudaSuccess) return err(PIVBOS_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    return PIVBOS_OK;
}
