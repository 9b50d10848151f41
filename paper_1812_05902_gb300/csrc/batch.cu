// Batched rendering and the autotuner (host side of include/pivbos.h's
// pivbos_batch_* and pivbos_autotune).  The persistent kernel lives in
// render.cu (batch_kernel), next to the single-render kernel it shares its
// per-chunk body with.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

struct pivbos_batch {
    int device;
    int integrator;
    pivbos_tuning tuning;
    int n_frames;
    std::vector<pivbos::BatchFrame> frames;   // in queue order
    std::vector<const double*> sources;       // per queued frame
    std::vector<uint32_t> n_src, n_pow2;
    std::vector<uint64_t*> keys;
    pivbos::BatchFrame* d_frames = nullptr;
    uint64_t* d_item_start = nullptr;
    unsigned long long* d_counter = nullptr;
    char* scratch = nullptr;
    uint64_t total_items = 0;
    int64_t kernels_per_run = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;   // private: the legacy default stream cannot be captured
};

namespace {

pivbos_status berr(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pivbos::set_last_error(buf);
    return st;
}

pivbos_status cerr(cudaError_t e, const char* what)
{
    return berr(e == cudaErrorMemoryAllocation ? PIVBOS_ERR_OOM : PIVBOS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool device_ptr(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

bool tuning_ok(const pivbos_tuning& t)
{
    return t.rays_per_cta >= 256 && t.rays_per_cta <= 2048 && t.rays_per_cta % 256 == 0 && t.ctas_per_sm >= 1 &&
           t.ctas_per_sm <= (t.cell_cache ? 2 : 3) && (t.cell_cache == 0 || t.cell_cache == 1);
}

int64_t sort_launches(uint32_t n_pow2)
{
    // morton keys, full shared sort, perm; per stage above 1024: global
    // merges for each stride >= 1024 and one shared merge
    int64_t k = 3;
    for (uint64_t st = 2048; st <= n_pow2; st <<= 1) {
        for (uint64_t j = st >> 1; j >= 1024; j >>= 1) ++k;
        ++k;
    }
    return k;
}

pivbos_status enqueue(pivbos_batch* b, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cerr(e, "batch queue reset");
    for (int f = 0; f < b->n_frames; ++f) {
        const pivbos::BatchFrame& F = b->frames[f];
        e = pivbos::launch_morton_sort(b->sources[f], b->n_src[f], b->keys[f], b->n_pow2[f],
                                       const_cast<uint32_t*>(F.p.perm), const_cast<float2*>(F.p.src_df), s);
        if (e != cudaSuccess) return cerr(e, "batch source ordering");
    }
    bool ext = false;
    for (int f = 0; f < b->n_frames; ++f) ext = ext || pivbos::optics_ext(b->frames[f].p.o);
    e = pivbos::launch_batch(b->d_frames, b->d_item_start, b->n_frames, b->total_items, b->d_counter, b->integrator,
                             b->tuning.cell_cache != 0, ext, b->tuning.ctas_per_sm, s);
    if (e != cudaSuccess) return cerr(e, "batch kernel");
    return PIVBOS_OK;
}

}  // namespace

extern "C" {

pivbos_status pivbos_default_tuning(pivbos_tuning* out)
{
    if (!out) return berr(PIVBOS_ERR_INVALID_ARG, "out is NULL");
    out->rays_per_cta = 2048;
    out->cell_cache = 0;
    out->ctas_per_sm = 3;
    out->use_graph = 1;
    return PIVBOS_OK;
}

pivbos_status pivbos_batch_create(const pivbos_frame_desc* frames, int n_frames, int integrator,
                                  const pivbos_tuning* tuning, pivbos_batch** out)
{
    pivbos::set_last_error("");
    if (!out) return berr(PIVBOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!frames || n_frames < 1) return berr(PIVBOS_ERR_INVALID_ARG, "no frames");
    pivbos_tuning t;
    pivbos_default_tuning(&t);
    if (tuning) t = *tuning;
    if (!tuning_ok(t)) return berr(PIVBOS_ERR_INVALID_ARG, "tuning out of range");
    std::vector<pivbos::BatchFrame> fr(n_frames);
    std::vector<double> cost(n_frames);
    int dev = -1;
    for (int f = 0; f < n_frames; ++f) {
        const pivbos_frame_desc& d = frames[f];
        int fdev = 0;
        uint64_t total = 0;
        memset(&fr[f], 0, sizeof(fr[f]));
        pivbos_status st = pivbos::prepare_trace(d.medium, d.optics, d.sources, d.n_sources, 1, d.rays_per_source,
                                                 d.seed, d.frame, integrator, d.step, &fr[f].p, &fdev, &total);
        if (st) {
            char msg[600];
            snprintf(msg, sizeof msg, "frame %d: %s", f, pivbos_last_error());
            pivbos::set_last_error(msg);
            return st;
        }
        if (!device_ptr(d.image, fdev)) return berr(PIVBOS_ERR_INVALID_ARG, "frame %d: image is not device memory", f);
        if (d.stats && !device_ptr(d.stats, fdev))
            return berr(PIVBOS_ERR_INVALID_ARG, "frame %d: stats is not device memory", f);
        dev = fdev;
        fr[f].image = d.image;
        fr[f].stats = d.stats;
        fr[f].rays_per_cta = (uint32_t)t.rays_per_cta;
        fr[f].total_rays = total;
        // estimated work: rays x (field evaluations expected per ray + fixed part)
        double evals = 0.0;
        if (d.medium) {
            const double depth = (double)(d.medium->n[2] - 1) * d.medium->spacing[2];
            evals = depth / d.step * (integrator == PIVBOS_RK4 ? 3.0 : 1.0);
        }
        cost[f] = (double)total * (30.0 + evals);
    }
    if (!tuning) {
        // without a tuning: the cell cache (and 2 CTAs per SM) when frames
        // whose geometry favours it (see the render's gather choice) carry
        // most of the estimated work
        double with = 0.0, all = 0.0;
        for (int f = 0; f < n_frames; ++f) {
            all += cost[f];
            if (fr[f].p.cell_cache) with += cost[f];
        }
        if (all > 0.0 && with >= 0.5 * all) {
            t.cell_cache = 1;
            t.ctas_per_sm = 2;
        }
    }
    for (int f = 0; f < n_frames; ++f) fr[f].p.cell_cache = t.cell_cache;
    pivbos_batch* b = new (std::nothrow) pivbos_batch();
    if (!b) return berr(PIVBOS_ERR_OOM, "host allocation");
    b->device = dev;
    b->integrator = integrator;
    b->tuning = t;
    b->n_frames = n_frames;
    std::vector<int> order(n_frames);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    // scratch per frame: keys | perm | double-float sources
    std::vector<size_t> off(n_frames);
    size_t bytes = 0;
    std::vector<uint64_t> item_start(n_frames + 1, 0);
    for (int q = 0; q < n_frames; ++q) {
        const int f = order[q];
        const uint32_t n = (uint32_t)frames[f].n_sources;
        uint32_t p2 = 2;
        while (p2 < n) p2 <<= 1;
        b->frames.push_back(fr[f]);
        b->sources.push_back(frames[f].sources);
        b->n_src.push_back(n);
        b->n_pow2.push_back(p2);
        off[q] = bytes;
        bytes += (size_t)p2 * 8 + (((size_t)n * 4 + 255) & ~(size_t)255) + (((size_t)n * 24 + 255) & ~(size_t)255);
        const uint64_t items = (fr[f].total_rays + t.rays_per_cta - 1) / t.rays_per_cta;
        item_start[q + 1] = item_start[q] + items;
        b->kernels_per_run += n > 0 ? sort_launches(p2) : 0;
    }
    b->kernels_per_run += 1;
    b->total_items = item_start[n_frames];
    cudaError_t e = cudaMalloc(&b->scratch, bytes > 0 ? bytes : 256);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_frames, sizeof(pivbos::BatchFrame) * n_frames);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_item_start, sizeof(uint64_t) * (n_frames + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        pivbos_batch_destroy(b);
        return cerr(e, "batch allocation");
    }
    for (int q = 0; q < n_frames; ++q) {
        char* base = b->scratch + off[q];
        const uint32_t n = b->n_src[q];
        b->keys.push_back((uint64_t*)base);
        b->frames[q].p.perm = (const uint32_t*)(base + (size_t)b->n_pow2[q] * 8);
        b->frames[q].p.src_df =
            (const float2*)(base + (size_t)b->n_pow2[q] * 8 + (((size_t)n * 4 + 255) & ~(size_t)255));
    }
    e = cudaMemcpy(b->d_frames, b->frames.data(), sizeof(pivbos::BatchFrame) * n_frames, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_item_start, item_start.data(), sizeof(uint64_t) * (n_frames + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pivbos_batch_destroy(b);
        return cerr(e, "batch upload");
    }
    *out = b;
    return PIVBOS_OK;
}

pivbos_status pivbos_batch_render(pivbos_batch* b, void* stream)
{
    pivbos::set_last_error("");
    if (!b) return berr(PIVBOS_ERR_INVALID_ARG, "batch is NULL");
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cerr(e, "cudaGetDevice");
    if (dev != b->device) return berr(PIVBOS_ERR_INVALID_ARG, "batch belongs to device %d", b->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (b->total_items == 0) return PIVBOS_OK;
    if (!b->tuning.use_graph) {
        const pivbos_status st = enqueue(b, s);
        return st;
    }
    if (!b->exec) {
        // capture once on a private stream; the instantiated graph is then
        // launched on whatever stream the caller passes
        if (!b->capture_stream) {
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cerr(e, "batch capture stream");
        }
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cerr(e, "batch capture");
        pivbos::timing_suppress(true);
        const pivbos_status st = enqueue(b, b->capture_stream);
        pivbos::timing_suppress(false);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->capture_stream, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cerr(e, "batch capture end");
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) return cerr(e, "batch graph instantiation");
        // the kernels were counted while capturing; replays count below
        pivbos::count_launches(-b->kernels_per_run);
    }
    e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cerr(e, "batch graph launch");
    pivbos::count_launches(b->kernels_per_run);
    return PIVBOS_OK;
}

void pivbos_batch_destroy(pivbos_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->scratch) cudaFree(b->scratch);
    if (b->d_frames) cudaFree(b->d_frames);
    if (b->d_item_start) cudaFree(b->d_item_start);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
static pivbos_status trace_sample(const pivbos_frame_desc* f, int integrator, double step, const int64_t* d_ids,
                                  int64_t n, pivbos_ray_state* d_out, std::vector<pivbos_ray_state>& host,
                                  cudaStream_t s)
{
    pivbos_status st = pivbos_trace_exit_states(f->medium, f->optics, f->sources, f->n_sources, 1,
                                                f->rays_per_source, f->seed, f->frame, integrator, step, d_ids, n,
                                                d_out, s);
    if (st) return st;
    host.resize(n);
    cudaError_t e = cudaMemcpyAsync(host.data(), d_out, sizeof(pivbos_ray_state) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cerr(e, "autotune sample read");
    return PIVBOS_OK;
}

static double sample_error(const std::vector<pivbos_ray_state>& a, const std::vector<pivbos_ray_state>& b)
{
    double err = 0.0;
    for (size_t q = 0; q < a.size(); ++q) {
        if (a[q].status != PIVBOS_RAY_REACHED || b[q].status != PIVBOS_RAY_REACHED) continue;
        err = fmax(err, fabs(a[q].sensor_xy[0] - b[q].sensor_xy[0]));
        err = fmax(err, fabs(a[q].sensor_xy[1] - b[q].sensor_xy[1]));
    }
    return err;
}

pivbos_status pivbos_autotune(const pivbos_frame_desc* frame, int integrator, double tol_px, int32_t n_sample_rays,
                              double* step_out, pivbos_tuning* tuning_out, void* stream)
{
    pivbos::set_last_error("");
    if (!frame || !step_out || !tuning_out) return berr(PIVBOS_ERR_INVALID_ARG, "NULL argument");
    if (!(tol_px > 0.0) || n_sample_rays < 1) return berr(PIVBOS_ERR_INVALID_ARG, "tol_px and n_sample_rays");
    if (integrator != PIVBOS_EULER && integrator != PIVBOS_RK4) return berr(PIVBOS_ERR_INVALID_ARG, "integrator");
    if (!(frame->step > 0.0)) return berr(PIVBOS_ERR_INVALID_ARG, "step");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = frame->n_sources * (int64_t)frame->rays_per_source;
    if (total <= 0) return berr(PIVBOS_ERR_INVALID_ARG, "frame has no rays");
    // ---- step ----
    double step = frame->step;
    if (frame->medium) {
        const int64_t n = std::min<int64_t>(n_sample_rays, total);
        std::vector<int64_t> ids(n);
        uint64_t x = 0x9E3779B97F4A7C15ull;   // fixed seeded sample (splitmix64 sequence)
        for (int64_t q = 0; q < n; ++q) {
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            ids[q] = (int64_t)(z % (uint64_t)total);
        }
        int64_t* d_ids = nullptr;
        pivbos_ray_state* d_out = nullptr;
        cudaError_t e = cudaMalloc(&d_ids, sizeof(int64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(pivbos_ray_state) * n);
        if (e == cudaSuccess) e = cudaMemcpy(d_ids, ids.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d_ids);
            cudaFree(d_out);
            return cerr(e, "autotune scratch");
        }
        const double richardson = integrator == PIVBOS_RK4 ? 16.0 / 15.0 : 2.0;
        std::vector<pivbos_ray_state> coarse, fine;
        auto err_of = [&](double h, double* err) -> pivbos_status {
            pivbos_status st = trace_sample(frame, integrator, h, d_ids, n, d_out, coarse, s);
            if (!st) st = trace_sample(frame, integrator, 0.5 * h, d_ids, n, d_out, fine, s);
            if (!st) *err = sample_error(coarse, fine) * richardson;
            return st;
        };
        double err = 0.0;
        pivbos_status st = err_of(step, &err);
        int guard = 0;
        while (!st && err > tol_px && guard++ < 6) {
            step *= 0.5;
            st = err_of(step, &err);
        }
        guard = 0;
        while (!st && err <= tol_px && guard++ < 6) {
            double e2 = 0.0;
            st = err_of(2.0 * step, &e2);
            if (st || e2 > tol_px) break;
            step *= 2.0;
            err = e2;
        }
        cudaFree(d_ids);
        cudaFree(d_out);
        if (st) return st;
    }
    *step_out = step;
    // ---- launch configuration ----
    pivbos_frame_desc sub = *frame;
    sub.step = step;
    const int64_t want = 4000000;
    sub.n_sources = std::max<int64_t>(1, std::min<int64_t>(frame->n_sources, want / std::max(1, frame->rays_per_source)));
    int H = frame->optics->d.H, W = frame->optics->d.W;
    int64_t* d_img = nullptr;
    cudaError_t e = cudaMalloc(&d_img, sizeof(int64_t) * (size_t)H * W);
    if (e != cudaSuccess) return cerr(e, "autotune image");
    sub.image = d_img;
    sub.stats = nullptr;
    cudaEvent_t a = nullptr, c = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&c);
    pivbos_tuning best;
    pivbos_default_tuning(&best);
    float best_ms = 1e30f;
    pivbos_status st = PIVBOS_OK;
    for (int cache = 0; cache <= 1 && !st; ++cache) {
        for (int rpc = 512; rpc <= 2048 && !st; rpc *= 2) {
            pivbos_tuning t;
            t.rays_per_cta = rpc;
            t.cell_cache = cache;
            t.ctas_per_sm = cache ? 2 : 3;
            t.use_graph = 0;
            pivbos_batch* b = nullptr;
            st = pivbos_batch_create(&sub, 1, integrator, &t, &b);
            if (st) break;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && !st; ++rep) {
                cudaEventRecord(a, s);
                st = pivbos_batch_render(b, s);
                cudaEventRecord(c, s);
                if (!st && cudaEventSynchronize(c) == cudaSuccess) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, c);
                    if (rep > 0) ms_min = std::min(ms_min, ms);
                }
            }
            pivbos_batch_destroy(b);
            if (!st && ms_min < best_ms) {
                best_ms = ms_min;
                best = t;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    cudaFree(d_img);
    if (st) return st;
    best.use_graph = 1;
    *tuning_out = best;
    return PIVBOS_OK;
}

}  // extern "C"
