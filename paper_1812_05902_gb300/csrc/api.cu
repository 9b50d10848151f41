// Host side of the pivbos C ABI (include/pivbos.h): handle lifetimes,
// argument checks, scratch memory, stream-ordered orchestration of the
// kernels, the device status word and kernel timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

namespace pivbos {
namespace {

thread_local std::string t_err;

pivbos_status fail(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

pivbos_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return fail(PIVBOS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PIVBOS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PV_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---- per-device status word ---------------------------------------------
// A file-scope device array: every device that loads the library holds its
// own copy, zero at load, so looking the word up never allocates (the render
// without allocation shares it).  Its host-side name is not a device
// address: the address is looked up once per device with that device current.
__device__ __align__(64) int g_status_word[16];

std::mutex g_dev_mu;
int* g_status[64] = {nullptr};

pivbos_status status_word(int dev, int** out)
{
    if (dev < 0 || dev >= 64) return fail(PIVBOS_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_status[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_status_word);
        if (e != cudaSuccess) return cuda_fail(e, "status word lookup");
        g_status[dev] = (int*)p;
    }
    *out = g_status[dev];
    return PIVBOS_OK;
}

// ---- kernel timing ----------------------------------------------------------
struct TimingRec {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimingRec> g_pending;
std::map<std::string, std::pair<double, int64_t>> g_totals;
thread_local long t_open = -1;
std::atomic<int64_t> g_launches{0};

// ---- checks -----------------------------------------------------------------
pivbos_status current_device(int* dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    return PIVBOS_OK;
}

// A pointer the caller declares as device memory must be device (or managed)
// memory of the current device: a host pointer handed to a kernel would fault.
pivbos_status check_device_ptr(const void* p, int dev, const char* what)
{
    if (!p) return fail(PIVBOS_ERR_INVALID_ARG, "%s is NULL", what);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PIVBOS_ERR_INVALID_ARG, "%s is not a CUDA pointer", what);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(PIVBOS_ERR_INVALID_ARG, "%s is not device memory", what);
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(PIVBOS_ERR_INVALID_ARG, "%s belongs to device %d, current is %d", what, a.device, dev);
    return PIVBOS_OK;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

dfc to_dfc(double v)
{
    const float hi = (float)v;
    return dfc{hi, (float)(v - (double)hi)};
}

uint32_t next_pow2(uint32_t v)
{
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// Rays per CTA of a render: PIVBOS_RAYS_PER_CTA if set, else 2048 in a
// dense medium (where a CTA reorders up to 2048 rays) and 256 otherwise (one
// ray per thread: warps stay close in stage, which eases instruction fetch;
// C1 5.51e9 -> 5.70e9 rays/s against 1024).
uint32_t rays_per_cta_setting(const TraceParams& p)
{
    // read once; a function-local static is initialised thread-safely
    static const long v = [] {
        const char* s = getenv("PIVBOS_RAYS_PER_CTA");
        const long x = s ? strtol(s, nullptr, 10) : 0;
        return (x >= 256 && x <= (1 << 20)) ? x : 0L;
    }();
    return v ? (uint32_t)v : (p.reorder ? 2048u : 256u);
}

// Gather strategy for a medium: reorder a CTA's rays when a ray makes many
// field evaluations (the box depth in steps times the stages per step); keep
// the last cell's corners in registers when, in addition, a step moves a ray
// by less than 0.75 of a grid spacing along every axis, so that consecutive
// stages mostly fall in one cell (PIVBOS_CELL_CACHE overrides).  Along z a
// step moves a ray by at most the step; across, by at most the step times
// the largest lateral slope of a ray that crosses the box toward the aim
// disk (the whole step when the aim disk is not beyond the box).
void choose_gather(const pivbos_medium* m, const pivbos_optics* o, double step, int integrator, TraceParams& p)
{
    const double evals = (double)(m->n[2] - 1) * m->spacing[2] / step * (integrator == PIVBOS_RK4 ? 3.0 : 1.0);
    p.reorder = evals >= 64.0 ? 1 : 0;
    double slope = 1.0;
    const double z_hi = m->origin[2] + (double)(m->n[2] - 1) * m->spacing[2];
    if (o && o->aim_z > z_hi) {
        double r = 0.0;
        for (int a = 0; a < 2; ++a)
            r = fmax(r, fmax(fabs(m->origin[a]), fabs(m->origin[a] + (double)(m->n[a] - 1) * m->spacing[a])));
        slope = fmin(1.0, (r + o->d.aim_r.hi) / (o->aim_z - z_hi));
    }
    const double move = fmax(step / m->spacing[2], fmax(step * slope / m->spacing[0], step * slope / m->spacing[1]));
    p.cell_cache = tuning_cell_cache(p.reorder && move < 0.75);
}

namespace {

// Common validation and parameter assembly for render / trace_exit_states.
struct Prepared {
    TraceParams p;
    int dev;
    uint64_t total;
};

pivbos_status prepare(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                      int64_t n_sources, int sources_on_device, int32_t rays_per_source, uint64_t seed,
                      uint32_t frame, int integrator, double step, Prepared* out)
{
    // argument checks that need no device come first
    if (!o) return fail(PIVBOS_ERR_INVALID_ARG, "optics handle is NULL");
    if (n_sources < 0 || rays_per_source < 0)
        return fail(PIVBOS_ERR_INVALID_ARG, "negative source or ray count");
    if (n_sources > 0 && !sources) return fail(PIVBOS_ERR_INVALID_ARG, "sources is NULL");
    if (integrator != PIVBOS_EULER && integrator != PIVBOS_RK4)
        return fail(PIVBOS_ERR_INVALID_ARG, "integrator %d", integrator);
    if (!finite_pos(step)) return fail(PIVBOS_ERR_INVALID_ARG, "step must be finite and > 0");
    const uint64_t total = (uint64_t)n_sources * (uint64_t)rays_per_source;
    if (n_sources > 0xffffffffll || total > (1ull << 31))
        return fail(PIVBOS_ERR_OVERFLOW, "%lld sources x %d rays exceeds 2^31 rays per render",
                    (long long)n_sources, rays_per_source);
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    if (o->device != dev) return fail(PIVBOS_ERR_INVALID_ARG, "optics handle belongs to device %d", o->device);
    if (m && m->device != dev) return fail(PIVBOS_ERR_INVALID_ARG, "medium handle belongs to device %d", m->device);
    if (n_sources > 0 && sources_on_device) {
        st = check_device_ptr(sources, dev, "sources");
        if (st) return st;
    }
    TraceParams& p = out->p;
    memset(&p, 0, sizeof p);
    if (m) {
        p.m.present = 1;
        p.m.field = m->field;
        double diag2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            p.m.n[a] = m->n[a];
            p.m.h[a] = (float)m->spacing[a];
            p.m.inv_h[a] = (float)(1.0 / m->spacing[a]);
            p.m.inv_hd[a] = to_dfc(1.0 / m->spacing[a]);
            p.m.origin[a] = to_dfc(m->origin[a]);
            p.m.lo[a] = to_dfc(m->origin[a]);
            p.m.hi[a] = to_dfc(m->origin[a] + (double)(m->n[a] - 1) * m->spacing[a]);
            const double L = (double)(m->n[a] - 1) * m->spacing[a];
            diag2 += L * L;
        }
        // step budget: twice the box diagonal in steps, plus four
        const double ms = ceil(2.0 * sqrt(diag2) / step) + 4.0;
        if (ms > 2.0e9) return fail(PIVBOS_ERR_UNSUPPORTED, "step too small for the box (%g steps)", ms);
        p.max_steps = (int)ms;
        p.m.z_key = (float)(m->origin[2] + 0.5 * (double)(m->n[2] - 1) * m->spacing[2]);
        choose_gather(m, o, step, integrator, p);
    }
    p.o = o->d;
    p.sources = sources;
    p.perm = nullptr;
    p.n_sources = (uint32_t)n_sources;
    p.rays_per_source = (uint32_t)rays_per_source;
    p.seed = seed;
    p.frame = frame;
    p.step = (float)step;
    p.step_d = step;
    p.step_df = to_dfc(step);
    st = status_word(dev, &p.status_word);
    if (st) return st;
    out->dev = dev;
    out->total = total;
    return PIVBOS_OK;
}

}  // namespace

void set_last_error(const char* msg) { t_err = msg; }

pivbos_status device_status_word(int dev, int** out) { return status_word(dev, out); }

pivbos_status failf(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

pivbos_status cuda_status(cudaError_t e, const char* what)
{
    return e == cudaSuccess ? PIVBOS_OK : cuda_fail(e, what);
}

pivbos_status device_pointer(const void* p, int dev, const char* what) { return check_device_ptr(p, dev, what); }

pivbos_status prepare_trace(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                            int64_t n_sources, int sources_on_device, int32_t rays_per_source, uint64_t seed,
                            uint32_t frame, int integrator, double step, TraceParams* p, int* dev, uint64_t* total)
{
    Prepared pr;
    const pivbos_status st = prepare(m, o, sources, n_sources, sources_on_device, rays_per_source, seed, frame,
                                     integrator, step, &pr);
    if (st) return st;
    *p = pr.p;
    *dev = pr.dev;
    *total = pr.total;
    return PIVBOS_OK;
}

bool g_timing_suppressed = false;
void timing_suppress(bool on) { g_timing_suppressed = on; }

int tuning_cell_cache(int dense)
{
    static const int v = [] {
        const char* s = getenv("PIVBOS_CELL_CACHE");
        return s ? (atoi(s) != 0 ? 1 : 0) : -1;
    }();
    return v >= 0 ? v : dense;
}

void timing_begin(const char* name, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_timing || g_timing_suppressed) return;
    TimingRec r;
    r.name = name;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    cudaEventRecord(r.a, s);
    g_pending.push_back(r);
    t_open = (long)g_pending.size() - 1;
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void timing_end(const char* name, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_timing || g_timing_suppressed || t_open < 0 || t_open >= (long)g_pending.size()) return;
    TimingRec& r = g_pending[t_open];
    if (r.name != name || r.b) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) return;
    cudaEventRecord(r.b, s);
    t_open = -1;
}

}  // namespace pivbos

using namespace pivbos;

extern "C" {

const char* pivbos_version(void) { return "pivbos 0.1 (sm_103a)"; }

int64_t pivbos_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* pivbos_last_error(void) { return t_err.c_str(); }

// ---------------------------------------------------------------------------
// medium
// ---------------------------------------------------------------------------
static pivbos_status medium_fill(pivbos_medium* m, const float* rho, int rho_on_device, cudaStream_t s)
{
    const int64_t N = (int64_t)m->n[0] * m->n[1] * m->n[2];
    const float* src = rho;
    if (!rho_on_device) {
        if (!m->rho_scratch) PV_CUDA(cudaMalloc(&m->rho_scratch, N * sizeof(float)), "rho staging allocation");
        PV_CUDA(cudaMemcpyAsync(m->rho_scratch, rho, N * sizeof(float), cudaMemcpyHostToDevice, s), "rho upload");
        src = m->rho_scratch;
    }
    PV_CUDA(launch_medium_prep(src, m->field, m->n[0], m->n[1], m->n[2], m->spacing, m->K, s), "medium_prep launch");
    return PIVBOS_OK;
}

pivbos_status pivbos_medium_create(const float* rho, int rho_on_device, int nx, int ny, int nz,
                                   const double origin[3], const double spacing[3], double K_GD,
                                   void* stream, pivbos_medium** out)
{
    t_err.clear();
    if (!out) return fail(PIVBOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!rho || !origin || !spacing) return fail(PIVBOS_ERR_INVALID_ARG, "rho, origin or spacing is NULL");
    if (nx < 2 || ny < 2 || nz < 2) return fail(PIVBOS_ERR_INVALID_ARG, "grid must have >= 2 nodes per axis");
    if ((int64_t)nx * ny * nz >= (1ll << 31) / 16)
        return fail(PIVBOS_ERR_UNSUPPORTED, "grid of %lld nodes is too large", (long long)nx * ny * nz);
    for (int a = 0; a < 3; ++a) {
        if (!finite_pos(spacing[a])) return fail(PIVBOS_ERR_INVALID_ARG, "spacing must be finite and > 0");
        if (!isfinite(origin[a])) return fail(PIVBOS_ERR_INVALID_ARG, "origin must be finite");
    }
    if (!isfinite(K_GD)) return fail(PIVBOS_ERR_INVALID_ARG, "K_GD must be finite");
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    if (rho_on_device) {
        st = check_device_ptr(rho, dev, "rho");
        if (st) return st;
    }
    pivbos_medium* m = new (std::nothrow) pivbos_medium();
    if (!m) return fail(PIVBOS_ERR_OOM, "host allocation");
    m->device = dev;
    m->n[0] = nx; m->n[1] = ny; m->n[2] = nz;
    for (int a = 0; a < 3; ++a) { m->origin[a] = origin[a]; m->spacing[a] = spacing[a]; }
    m->K = K_GD;
    const int64_t N = (int64_t)nx * ny * nz;
    cudaError_t e = cudaMalloc(&m->field, N * sizeof(float4));
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "field allocation");
    }
    st = medium_fill(m, rho, rho_on_device, (cudaStream_t)stream);
    if (st) {
        pivbos_medium_destroy(m);
        return st;
    }
    *out = m;
    return PIVBOS_OK;
}

pivbos_status pivbos_medium_refill(pivbos_medium* m, const float* rho, int rho_on_device, void* stream)
{
    t_err.clear();
    if (!m || !rho) return fail(PIVBOS_ERR_INVALID_ARG, "medium or rho is NULL");
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    if (m->device != dev) return fail(PIVBOS_ERR_INVALID_ARG, "medium belongs to device %d", m->device);
    if (rho_on_device) {
        st = check_device_ptr(rho, dev, "rho");
        if (st) return st;
    }
    st = medium_fill(m, rho, rho_on_device, (cudaStream_t)stream);
    if (st == PIVBOS_OK) ++m->version;
    return st;
}

void pivbos_medium_destroy(pivbos_medium* m)
{
    if (!m) return;
    // cudaFree waits for work on the device that may still read the field
    if (m->field) cudaFree(m->field);
    if (m->rho_scratch) cudaFree(m->rho_scratch);
    delete m;
}

// ---------------------------------------------------------------------------
// optics
// ---------------------------------------------------------------------------
pivbos_status pivbos_optics_create(const pivbos_surface* surfaces, int n_surfaces, double n_object,
                                   double aim_z, double aim_radius, double f_number, double magnification,
                                   double wavelength, int dtau_rule, double sensor_z, double pixel_pitch,
                                   int width, int height, pivbos_optics** out)
{
    t_err.clear();
    if (!out) return fail(PIVBOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_surfaces < 0 || n_surfaces > PIVBOS_MAX_SURFACES)
        return fail(PIVBOS_ERR_INVALID_ARG, "n_surfaces %d outside [0, %d]", n_surfaces, PIVBOS_MAX_SURFACES);
    if (n_surfaces > 0 && !surfaces) return fail(PIVBOS_ERR_INVALID_ARG, "surfaces is NULL");
    if (!finite_pos(n_object)) return fail(PIVBOS_ERR_INVALID_ARG, "n_object must be > 0");
    if (!isfinite(aim_z) || !(isfinite(aim_radius) && aim_radius >= 0.0))
        return fail(PIVBOS_ERR_INVALID_ARG, "aim disk must be finite");
    if (!finite_pos(f_number) || !(isfinite(magnification) && magnification >= 0.0) || !finite_pos(wavelength))
        return fail(PIVBOS_ERR_INVALID_ARG, "f_number, magnification, wavelength");
    if (dtau_rule != 0 && dtau_rule != 1) return fail(PIVBOS_ERR_INVALID_ARG, "dtau_rule %d", dtau_rule);
    if (!isfinite(sensor_z) || !finite_pos(pixel_pitch)) return fail(PIVBOS_ERR_INVALID_ARG, "sensor");
    if (width < 1 || height < 1 || (int64_t)width * height > (1ll << 30))
        return fail(PIVBOS_ERR_INVALID_ARG, "sensor %d x %d", width, height);
    for (int i = 0; i < n_surfaces; ++i) {
        const pivbos_surface& s = surfaces[i];
        if (s.type < PIVBOS_SURF_SPHERE || s.type > PIVBOS_SURF_LENS_ARRAY || s.reserved != 0 ||
            !isfinite(s.z_vertex) || !isfinite(s.radius) || !(isfinite(s.clear_radius) && s.clear_radius >= 0.0) ||
            ((s.type == PIVBOS_SURF_SPHERE || s.type == PIVBOS_SURF_PLANE) && !finite_pos(s.n_after)) ||
            ((s.type == PIVBOS_SURF_IDEAL_THIN || s.type == PIVBOS_SURF_LENS_ARRAY) &&
             !(isfinite(s.focal) && s.focal != 0.0)) ||
            (s.type == PIVBOS_SURF_LENS_ARRAY && !(s.radius > 0.0)))
            return fail(PIVBOS_ERR_INVALID_ARG, "surface %d is malformed", i);
    }
    {
        const double dtau = 2.44 * (dtau_rule == 0 ? M_PI : 1.0) * f_number * (magnification + 1.0) * wavelength;
        const double sp = dtau / 4.0 / pixel_pitch;
        if (!(sp > 0.0) || sp > (PIVBOS_MAX_WINDOW - 2) / 6.0)
            return fail(PIVBOS_ERR_UNSUPPORTED, "spot sigma %.3g px outside (0, %.3g]", sp,
                        (PIVBOS_MAX_WINDOW - 2) / 6.0);
    }
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    pivbos_optics* o = new (std::nothrow) pivbos_optics();
    if (!o) return fail(PIVBOS_ERR_OOM, "host allocation");
    o->device = dev;
    DevOptics& d = o->d;
    memset(&d, 0, sizeof d);
    d.ns = n_surfaces;
    double n_cur = n_object;
    for (int i = 0; i < n_surfaces; ++i) {
        const pivbos_surface& s = surfaces[i];
        DevSurface& D = d.s[i];
        // a sphere of zero radius is a flat refracting surface
        D.type = (s.type == PIVBOS_SURF_SPHERE && s.radius == 0.0) ? PIVBOS_SURF_PLANE : s.type;
        D.R_f = (float)s.radius;
        D.clear_r2 = (float)(s.clear_radius * s.clear_radius);
        D.z = to_dfc(s.z_vertex);
        D.R = to_dfc(s.radius);
        D.invR = to_dfc(s.radius != 0.0 ? 1.0 / s.radius : 0.0);
        D.inv_f = to_dfc((s.type == PIVBOS_SURF_IDEAL_THIN || s.type == PIVBOS_SURF_LENS_ARRAY) ? 1.0 / s.focal
                                                                                               : 0.0);
        if (D.type == PIVBOS_SURF_SPHERE || D.type == PIVBOS_SURF_PLANE) {
            const double eta = n_cur / s.n_after;
            D.eta = to_dfc(eta);
            D.eta2 = to_dfc(eta * eta);
            n_cur = s.n_after;
        }
    }
    d.W = width;
    d.H = height;
    d.aim_z = to_dfc(aim_z);
    d.aim_r = to_dfc(aim_radius);
    const double dtau = 2.44 * (dtau_rule == 0 ? M_PI : 1.0) * f_number * (magnification + 1.0) * wavelength;
    const double sigma = dtau / 4.0;
    const double sp = sigma / pixel_pitch;
    d.sigma_px = (float)sp;
    d.win3 = (float)(3.0 * sp);
    d.inv_sqrt2_sigma = (float)(1.0 / (M_SQRT2 * sp));
    d.sensor_z = to_dfc(sensor_z);
    d.inv_pitch = to_dfc(1.0 / pixel_pitch);
    d.half_w = 0.5f * (float)width;
    d.half_h = 0.5f * (float)height;
    o->aim_z = aim_z;
    o->magnification = magnification;
    o->n_object = n_object;
    o->pixel_pitch = pixel_pitch;
    *out = o;
    return PIVBOS_OK;
}

pivbos_status pivbos_optics_tilt_sensor(const pivbos_optics* o, double tilt_x, double tilt_y, pivbos_optics** out)
{
    t_err.clear();
    if (!o || !out) return fail(PIVBOS_ERR_INVALID_ARG, "optics or out is NULL");
    *out = nullptr;
    if (!isfinite(tilt_x) || !isfinite(tilt_y)) return fail(PIVBOS_ERR_INVALID_ARG, "tilt angles must be finite");
    pivbos_optics* c = new (std::nothrow) pivbos_optics(*o);
    if (!c) return fail(PIVBOS_ERR_OOM, "host allocation");
    c->rad_owned = nullptr;
    if (o->rad_owned) {
        // the copy owns a copy of the radiance table
        float2* t = nullptr;
        cudaError_t e = cudaMalloc((void**)&t, (size_t)o->d.rad_n * sizeof(float2));
        if (e == cudaSuccess)
            e = cudaMemcpy(t, o->rad_owned, (size_t)o->d.rad_n * sizeof(float2), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            if (t) cudaFree(t);
            delete c;
            return cuda_fail(e, "radiance table copy");
        }
        c->rad_owned = t;
        c->d.rad = t;
    }
    // the sensor's axes: x, y, z turned by tilt_x about x, then by tilt_y about y
    const double cx = cos(tilt_x), sx = sin(tilt_x), cy = cos(tilt_y), sy = sin(tilt_y);
    const double eu[3] = {cy, 0.0, -sy};
    const double ev[3] = {sy * sx, cx, cy * sx};
    const double en[3] = {sy * cx, -sx, cy * cx};
    DevOptics& d = c->d;
    d.tilted = 1;
    for (int a = 0; a < 3; ++a) {
        d.eu[a] = to_dfc(eu[a]);
        d.ev[a] = to_dfc(ev[a]);
        d.en[a] = to_dfc(en[a]);
    }
    *out = c;
    return PIVBOS_OK;
}

void pivbos_optics_destroy(pivbos_optics* o)
{
    if (!o) return;
    // cudaFree waits for work on the device that may still read the table
    if (o->rad_owned) cudaFree(o->rad_owned);
    delete o;
}

// ---------------------------------------------------------------------------
// render
// ---------------------------------------------------------------------------
static pivbos_status render_impl(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                                 int64_t n_sources, int64_t first_source, int sources_on_device,
                                 int32_t rays_per_source, uint64_t seed, uint32_t frame, int integrator, double step,
                                 int64_t* image, int image_on_device, int64_t* stats, void* stream);

pivbos_status pivbos_render(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                            int64_t n_sources, int sources_on_device, int32_t rays_per_source, uint64_t seed,
                            uint32_t frame, int integrator, double step, int64_t* image, int image_on_device,
                            int64_t* stats, void* stream)
{
    return render_impl(m, o, sources, n_sources, 0, sources_on_device, rays_per_source, seed, frame, integrator,
                       step, image, image_on_device, stats, stream);
}

pivbos_status pivbos_render_range(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                                  int64_t n_sources, int64_t first_source, int sources_on_device,
                                  int32_t rays_per_source, uint64_t seed, uint32_t frame, int integrator,
                                  double step, int64_t* image, int image_on_device, int64_t* stats, void* stream)
{
    t_err.clear();
    if (first_source < 0 || first_source + n_sources > 0xffffffffll)
        return fail(PIVBOS_ERR_INVALID_ARG, "first_source %lld outside [0, 2^32 - n_sources]", (long long)first_source);
    return render_impl(m, o, sources, n_sources, first_source, sources_on_device, rays_per_source, seed, frame,
                       integrator, step, image, image_on_device, stats, stream);
}

static pivbos_status render_impl(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                                 int64_t n_sources, int64_t first_source, int sources_on_device,
                                 int32_t rays_per_source, uint64_t seed, uint32_t frame, int integrator, double step,
                                 int64_t* image, int image_on_device, int64_t* stats, void* stream)
{
    t_err.clear();
    if (!image) return fail(PIVBOS_ERR_INVALID_ARG, "image is NULL");
    Prepared pr;
    pivbos_status st = prepare(m, o, sources, n_sources, sources_on_device, rays_per_source, seed, frame,
                               integrator, step, &pr);
    if (st) return st;
    if (image_on_device) {
        st = check_device_ptr(image, pr.dev, "image");
        if (st) return st;
    }
    if (stats) {
        st = check_device_ptr(stats, pr.dev, "stats");
        if (st) return st;
    }
    if (pr.total == 0) return PIVBOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)n_sources;
    const uint32_t n_pow2 = next_pow2(n < 2 ? 2 : n);
    const size_t img_bytes = (size_t)o->d.W * o->d.H * sizeof(int64_t);
    // scratch: keys | perm | double-float sources | sources copy | image copy
    const size_t off_perm = (size_t)n_pow2 * 8;
    const size_t off_sdf = off_perm + (((size_t)n * 4 + 255) & ~(size_t)255);
    const size_t off_src = off_sdf + (((size_t)n * 24 + 255) & ~(size_t)255);
    const size_t off_img = off_src + (sources_on_device ? 0 : (((size_t)n * 24 + 255) & ~(size_t)255));
    const size_t bytes = off_img + (image_on_device ? 0 : img_bytes);
    char* scratch = nullptr;
    PV_CUDA(cudaMallocAsync((void**)&scratch, bytes, s), "render scratch allocation");
    uint64_t* keys = (uint64_t*)scratch;
    uint32_t* perm = (uint32_t*)(scratch + off_perm);
    float2* sdf = (float2*)(scratch + off_sdf);
    const double* dsrc = sources;
    int64_t* dimg = image;
    cudaError_t e = cudaSuccess;
    if (!sources_on_device) {
        e = cudaMemcpyAsync(scratch + off_src, sources, (size_t)n * 24, cudaMemcpyHostToDevice, s);
        dsrc = (const double*)(scratch + off_src);
    }
    if (e == cudaSuccess && !image_on_device) {
        dimg = (int64_t*)(scratch + off_img);
        e = cudaMemcpyAsync(dimg, image, img_bytes, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = launch_morton_sort(dsrc, n, keys, n_pow2, perm, sdf, s);
    if (e == cudaSuccess) {
        pr.p.sources = dsrc;
        pr.p.perm = perm;
        pr.p.src_df = sdf;
        pr.p.source_offset = (uint32_t)first_source;
        e = launch_render(pr.p, integrator, dimg, stats, rays_per_cta_setting(pr.p), s);
    }
    if (e == cudaSuccess && !image_on_device)
        e = cudaMemcpyAsync(image, dimg, img_bytes, cudaMemcpyDeviceToHost, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "render");
    if (ef != cudaSuccess) return cuda_fail(ef, "render scratch release");
    if (!image_on_device) PV_CUDA(cudaStreamSynchronize(s), "render (host image) synchronisation");
    return PIVBOS_OK;
}

pivbos_status pivbos_trace_exit_states(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                                       int64_t n_sources, int sources_on_device, int32_t rays_per_source,
                                       uint64_t seed, uint32_t frame, int integrator, double step,
                                       const int64_t* ray_ids, int64_t n_rays, pivbos_ray_state* out,
                                       void* stream)
{
    t_err.clear();
    Prepared pr;
    pivbos_status st = prepare(m, o, sources, n_sources, sources_on_device, rays_per_source, seed, frame,
                               integrator, step, &pr);
    if (st) return st;
    if (n_rays < 0) return fail(PIVBOS_ERR_INVALID_ARG, "n_rays < 0");
    if (n_rays == 0) return PIVBOS_OK;
    if (!ray_ids && (uint64_t)n_rays > pr.total)
        return fail(PIVBOS_ERR_INVALID_ARG, "n_rays exceeds the rays of the render");
    st = check_device_ptr(out, pr.dev, "out");
    if (st) return st;
    if (ray_ids) {
        st = check_device_ptr(ray_ids, pr.dev, "ray_ids");
        if (st) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double* dsrc = sources;
    void* scratch = nullptr;
    if (!sources_on_device) {
        PV_CUDA(cudaMallocAsync(&scratch, (size_t)n_sources * 24, s), "trace scratch allocation");
        cudaError_t e = cudaMemcpyAsync(scratch, sources, (size_t)n_sources * 24, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(scratch, s);
            return cuda_fail(e, "sources upload");
        }
        dsrc = (const double*)scratch;
    }
    pr.p.sources = dsrc;
    cudaError_t e = launch_trace_states(pr.p, integrator, ray_ids, n_rays, out, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "trace_exit_states");
    return PIVBOS_OK;
}

pivbos_status pivbos_image_finalize(const int64_t* image, int64_t n_pixels, float* out, void* stream)
{
    t_err.clear();
    if (n_pixels < 0) return fail(PIVBOS_ERR_INVALID_ARG, "n_pixels < 0");
    if (n_pixels == 0) return PIVBOS_OK;
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    st = check_device_ptr(image, dev, "image");
    if (st) return st;
    st = check_device_ptr(out, dev, "out");
    if (st) return st;
    PV_CUDA(launch_finalize(image, n_pixels, out, (cudaStream_t)stream), "finalize");
    return PIVBOS_OK;
}

pivbos_status pivbos_sync(void* stream)
{
    t_err.clear();
    int dev;
    pivbos_status st = current_device(&dev);
    if (st) return st;
    PV_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronisation");
    int* sw = nullptr;
    st = status_word(dev, &sw);
    if (st) return st;
    int v = 0;
    PV_CUDA(cudaMemcpy(&v, sw, sizeof v, cudaMemcpyDeviceToHost), "status word read");
    if (v != 0) {
        PV_CUDA(cudaMemset(sw, 0, sizeof v), "status word clear");
        return fail((pivbos_status)v, "device reported status %d", v);
    }
    return PIVBOS_OK;
}

pivbos_status pivbos_timing_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = on != 0;
    return PIVBOS_OK;
}

static void drain_pending_locked()
{
    for (auto& r : g_pending) {
        if (r.a && r.b) {
            float ms = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                auto& t = g_totals[r.name];
                t.first += ms;
                t.second += 1;
            }
        }
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    g_pending.clear();
}

pivbos_status pivbos_timing_reset(void)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    drain_pending_locked();
    g_totals.clear();
    return PIVBOS_OK;
}

pivbos_status pivbos_timing_read(const char* prefix, double* ms_total, int64_t* launches)
{
    if (!prefix || !ms_total || !launches) return fail(PIVBOS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g_tmu);
    drain_pending_locked();
    double ms = 0.0;
    int64_t n = 0;
    const size_t lp = strlen(prefix);
    for (auto& kv : g_totals) {
        if (kv.first.compare(0, lp, prefix) == 0) {
            ms += kv.second.first;
            n += kv.second.second;
        }
    }
    *ms_total = ms;
    *launches = n;
    return PIVBOS_OK;
}

}  // extern "C"
