// The learned ray map (surrogate): host API of the MLP test hooks and of
// training / rendering with the surrogate.  The network maps a ray's entry
// state to the residual of its exit line (the paper has no learned part;
// this is a library facility built on the same tracer).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "handles.cuh"
#include "mlp.cuh"

namespace {

pivbos_status serr(pivbos_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pivbos::set_last_error(buf);
    return st;
}

pivbos_status scuda(cudaError_t e, const char* what)
{
    return serr(e == cudaErrorMemoryAllocation ? PIVBOS_ERR_OOM : PIVBOS_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

}  // namespace

#include "surrogate_kernels.cuh"

namespace pivbos {

// The network over a served list (one persistent CTA per SM, two
// warpgroups each): R = B + MLP(X) * t_scale.  The render and the
// per-element check of the testing library both launch it through here.
cudaError_t launch_surr_net(const SurrParams& S, const __nv_bfloat16* wbf, const float* params, const ServedList& sv,
                            int* status_word, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // per device, so set on every launch (cheap)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(surr_net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(NetSmem));
    if (e != cudaSuccess) return e;
    timing_begin("surrogate_net", s);
    surr_net_kernel<<<sms, 128 * kNetGroups, sizeof(NetSmem), s>>>(S, wbf, params, sv, status_word);
    timing_end("surrogate_net", s);
    count_launches(1);
    return cudaGetLastError();
}

// For the per-element check of the network kernel: n rows of inputs X
// (BF16 [n][16], device), projection residuals B (device float4 [n]) and the
// output scales; writes R (device float4 [n]).  Synchronous.
cudaError_t surr_net_apply(const MlpDev& net, const __nv_bfloat16* X, const float4* B, const float t_scale[4],
                           uint32_t n, float4* R, int* timed_out, cudaStream_t s)
{
    SurrParams S;
    memset(&S, 0, sizeof S);
    for (int q = 0; q < 4; ++q) S.t_scale[q] = t_scale[q];
    unsigned long long* count = nullptr;
    int* status = nullptr;
    cudaError_t e = cudaMalloc(&count, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    const unsigned long long nn = n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, &nn, sizeof nn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
    ServedList sv;
    memset(&sv, 0, sizeof sv);
    sv.X = const_cast<__nv_bfloat16*>(X);
    sv.B = const_cast<float4*>(B);
    sv.R = R;
    sv.count = count;
    sv.capacity = n;
    if (e == cudaSuccess) e = launch_surr_net(S, net.wbf, net.params, sv, status, s);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *timed_out = st != 0;
    cudaFree(count);
    cudaFree(status);
    return e;
}

}  // namespace pivbos

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#include <chrono>

struct pivbos_surrogate {
    int device = 0;
    int integrator = PIVBOS_RK4;
    const pivbos_medium* medium = nullptr;
    uint64_t medium_version = 0;   // the medium's version when trained
    const pivbos_optics* optics = nullptr;
    pivbos::MlpDev net;
    pivbos::SurrParams S;
    uint32_t* bin_ok = nullptr;
    uint32_t* bin_net = nullptr;
    float4* table = nullptr;
    pivbos_surrogate_report rep;
};

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

pivbos::dfc to_dfc2(double v)
{
    const float hi = (float)v;
    return pivbos::dfc{hi, (float)(v - (double)hi)};
}

// He-uniform initial weights (bound sqrt(6/in)), zero biases; splitmix64.
void init_params(std::vector<float>& p, uint64_t seed)
{
    p.assign(pivbos::kMlpParams, 0.f);
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < pivbos::kMlpLayers; ++l) {
        const int in = pivbos::mlp_in(l), out = pivbos::mlp_out(l);
        const double bound = sqrt(6.0 / in);
        for (int e = 0; e < in * out; ++e) p[pivbos::mlp_w_offset(l) + e] = (float)((2.0 * next() - 1.0) * bound);
    }
}

template <typename T>
struct DevBuf {
    T* p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * (n > 0 ? n : 1)); }
    ~DevBuf() { cudaFree(p); }
};

// Greedy choice of served bins under a global error budget: bins in order of
// plain-path work saved per unit of squared error, while the summed squared
// error stays within budget2 (all in held-out sums).  Returns the served
// bins' error, steps and ray count.
struct Served {
    double err2 = 0.0, steps = 0.0, rays = 0.0;
};

Served choose_bins(const std::vector<double>& err2, const std::vector<double>& steps,
                   const std::vector<unsigned>& cnt, int min_count, double budget2, std::vector<uint32_t>* ok)
{
    std::vector<int> order;
    for (int b = 0; b < (int)cnt.size(); ++b)
        if ((int)cnt[b] >= min_count) order.push_back(b);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        // steps[a] / err2[a] > steps[b] / err2[b], without dividing by zero
        const double l = steps[a] * err2[b], r = steps[b] * err2[a];
        return l != r ? l > r : a < b;
    });
    Served sv;
    for (int b : order) {
        if (sv.err2 + err2[b] > budget2) continue;
        sv.err2 += err2[b];
        sv.steps += steps[b];
        sv.rays += cnt[b];
        if (ok) (*ok)[b >> 5] |= 1u << (b & 31);
    }
    return sv;
}

// Automatic mode trains the network when the projection alone, served
// within the budget, saves less than this share of the plain path's steps.
constexpr double kAutoTrainBelow = 0.99;

// Render cost of a held-out ray by how it is served, in units of one plain
// integration step of one ray, measured on GB300 (C4: a plain step 18 ps; a
// ray served by the projection alone in the direct pass 83.5 ps with 1
// segment, 465 ps with 32; the network's forward 95 ps more; a plain
// fallback ray its steps plus ~120 ps of generation, optics and deposit).
inline double cost_projection(int segments) { return 3.9 + 0.68 * segments; }
constexpr double kCostNetworkExtra = 5.3;
constexpr double kCostFallbackRay = 7.0;
// A plan whose bins take no network renders its served rays in one direct
// pass, without the served list and the separate finish kernel a plan with
// the network needs: about 1.5 plain steps cheaper per served ray (C4 with
// one projection segment: 83.5 ms against prep + finish 110.0 ms per 1e9
// rays, at ~18 ps per plain RK4 step).
constexpr double kCostListRay = 1.5;

struct Mixed {
    double err2 = 0.0, steps = 0.0, rays = 0.0, net_rays = 0.0, cost = 0.0;
};

// Per-bin choice among the projection alone (err2p), the projection with the
// network's correction (err2n) and the plain fallback (no error): for a
// multiplier lam, every bin takes the option of least cost + lam * err2;
// lam is the smallest (bisected) whose summed error meets budget2, which
// minimises the render cost under the budget up to the bins' granularity.
// Bins with fewer than min_count held-out rays fall back.  with_net false
// leaves the network out (the projection alone or the fallback per bin).
Mixed choose_mixed(const std::vector<double>& err2n, const std::vector<double>& err2p,
                   const std::vector<double>& steps, const std::vector<unsigned>& cnt, int min_count, double budget2,
                   int segments, bool with_net, std::vector<uint32_t>* ok, std::vector<uint32_t>* net)
{
    const int nb = (int)cnt.size();
    const double kCostProjection = cost_projection(segments), kCostNetwork = kCostProjection + kCostNetworkExtra;
    auto pick = [&](double lam, bool write) {
        Mixed m;
        for (int b = 0; b < nb; ++b) {
            const double n = cnt[b];
            if (cnt[b] == 0) continue;
            const double fb = steps[b] + kCostFallbackRay * n;
            int choice = 0;   // 0 fallback, 1 projection, 2 network
            double best = fb;
            if ((int)cnt[b] >= min_count) {
                const double cp = kCostProjection * n + lam * err2p[b];
                const double cn = kCostNetwork * n + lam * err2n[b];
                if (cp < best) { best = cp; choice = 1; }
                if (with_net && cn < best) { best = cn; choice = 2; }
            }
            if (choice == 0) {
                m.cost += fb;
                continue;
            }
            m.err2 += choice == 2 ? err2n[b] : err2p[b];
            m.cost += (choice == 2 ? kCostNetwork : kCostProjection) * n;
            m.steps += steps[b];
            m.rays += n;
            if (choice == 2) m.net_rays += n;
            if (write) {
                (*ok)[b >> 5] |= 1u << (b & 31);
                if (choice == 2) (*net)[b >> 5] |= 1u << (b & 31);
            }
        }
        return m;
    };
    double lam = 0.0;
    if (pick(0.0, false).err2 > budget2) {
        double lo = 0.0, hi = 1.0;
        while (pick(hi, false).err2 > budget2 && hi < 1e300) hi *= 16.0;
        for (int it = 0; it < 200; ++it) {
            const double mid = lo > 0.0 ? sqrt(lo * hi) : hi / 16.0;
            if (pick(mid, false).err2 > budget2) lo = mid;
            else hi = mid;
            if (lo > 0.0 && hi / lo < 1.0 + 1e-12) break;
        }
        lam = hi;
    }
    Mixed m = pick(lam, true);
    // The bins are coarse, so one multiplier can leave part of the budget
    // unused: serve further fallback bins, in order of cost saved per unit of
    // squared error, with whichever predictor saves the most and still fits.
    struct Up { double ratio, save, e2; int b, choice; };
    std::vector<Up> ups;
    for (int b = 0; b < nb; ++b) {
        if ((int)cnt[b] < min_count || (((*ok)[b >> 5] >> (b & 31)) & 1u)) continue;
        const double n = cnt[b], fb = steps[b] + kCostFallbackRay * n;
        const double sp = fb - kCostProjection * n, sn = fb - kCostNetwork * n;
        if (sp > 0.0) ups.push_back({sp / fmax(err2p[b], 1e-300), sp, err2p[b], b, 1});
        if (with_net && sn > 0.0) ups.push_back({sn / fmax(err2n[b], 1e-300), sn, err2n[b], b, 2});
    }
    std::sort(ups.begin(), ups.end(), [](const Up& x, const Up& y) {
        return x.ratio != y.ratio ? x.ratio > y.ratio : (x.b != y.b ? x.b < y.b : x.choice < y.choice);
    });
    for (const Up& u : ups) {
        if (((*ok)[u.b >> 5] >> (u.b & 31)) & 1u) continue;   // served by an earlier candidate
        if (m.err2 + u.e2 > budget2) continue;
        const double n = cnt[u.b];
        m.err2 += u.e2;
        m.cost -= u.save;
        m.steps += steps[u.b];
        m.rays += n;
        (*ok)[u.b >> 5] |= 1u << (u.b & 31);
        if (u.choice == 2) {
            m.net_rays += n;
            (*net)[u.b >> 5] |= 1u << (u.b & 31);
        }
    }
    return m;
}

}  // namespace

namespace pivbos {

// The per-bin plan of choose_mixed for the testing library (host code; its
// declaration is in testing.cu): ok and net are n_bins / 32 words of bits;
// returns the plan's cost in plain steps.
double plan_bins(const double* err2n, const double* err2p, const double* steps, const unsigned* cnt, int n_bins,
                 int min_count, double budget2, int segments, bool with_net, uint32_t* ok, uint32_t* net,
                 double* err2_out, double* rays_out, double* net_rays_out)
{
    const std::vector<double> en(err2n, err2n + n_bins), ep(err2p, err2p + n_bins), st(steps, steps + n_bins);
    const std::vector<unsigned> c(cnt, cnt + n_bins);
    std::vector<uint32_t> okv((size_t)n_bins / 32, 0u), netv((size_t)n_bins / 32, 0u);
    const Mixed m = choose_mixed(en, ep, st, c, min_count, budget2, segments, with_net, &okv, &netv);
    std::copy(okv.begin(), okv.end(), ok);
    std::copy(netv.begin(), netv.end(), net);
    *err2_out = m.err2;
    *rays_out = m.rays;
    *net_rays_out = m.net_rays;
    return m.cost;
}

}  // namespace pivbos

extern "C" {

pivbos_status pivbos_surrogate_default_cfg(pivbos_surrogate_cfg* c)
{
    if (!c) return serr(PIVBOS_ERR_INVALID_ARG, "cfg is NULL");
    c->n_train = 20000000;
    c->n_val = 2000000;
    // 5 passes over 2e7 rays: on C4 at 0.001 px the served fraction of 20
    // passes (99.86 %) at a quarter of the time (1.6 s on GB300)
    c->epochs = 5;
    c->batch = 16384;
    c->lr = 3e-3f;
    c->err_budget_px = 0.01f;
    c->budget_margin = 0.8f;
    c->min_bin_count = 8;
    c->seed = 7;
    c->ref_plane_z = NAN;
    c->born_segments = -1;
    c->use_network = -1;
    c->table_columns_per_cell = 0;
    c->table_levels_per_cell = 1;
    return PIVBOS_OK;
}

pivbos_status pivbos_surrogate_train(const pivbos_frame_desc* frame, int integrator, const pivbos_surrogate_cfg* cfg,
                                     pivbos_surrogate** out, pivbos_surrogate_report* report, void* stream)
{
    pivbos::set_last_error("");
    if (!frame || !out) return serr(PIVBOS_ERR_INVALID_ARG, "frame and out are required");
    *out = nullptr;
    if (!frame->medium) return serr(PIVBOS_ERR_INVALID_ARG, "the surrogate needs a medium");
    pivbos_surrogate_cfg c;
    pivbos_surrogate_default_cfg(&c);
    if (cfg) c = *cfg;
    if (c.n_train < 256 || c.n_val < 256 || c.n_train > (1ll << 31) || c.n_val > (1ll << 31) || c.epochs < 1 ||
        c.batch < 256 || c.batch > 65536 || !(c.lr > 0.f) || !(c.err_budget_px > 0.f) ||
        !(c.budget_margin > 0.f && c.budget_margin <= 1.f) || c.min_bin_count < 1 ||
        (!std::isnan(c.ref_plane_z) && !std::isfinite(c.ref_plane_z)) ||
        c.born_segments < -1 || c.born_segments > 64 || (c.use_network < -1 || c.use_network > 1) ||
        c.table_columns_per_cell < 0 || c.table_columns_per_cell > 8 || c.table_levels_per_cell < 1 ||
        c.table_levels_per_cell > 4)
        return serr(PIVBOS_ERR_INVALID_ARG, "surrogate configuration out of range");
    pivbos::TraceParams P;
    int dev = 0;
    uint64_t total = 0;
    pivbos_status st = pivbos::prepare_trace(frame->medium, frame->optics, frame->sources, frame->n_sources, 1,
                                             frame->rays_per_source, frame->seed, frame->frame, integrator, frame->step,
                                             &P, &dev, &total);
    if (st) return st;
    if (total == 0) return serr(PIVBOS_ERR_INVALID_ARG, "frame has no rays");
    cudaStream_t s = (cudaStream_t)stream;
    const pivbos_medium* m = frame->medium;
    const pivbos_optics* o = frame->optics;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = m->origin[a];
        hi[a] = m->origin[a] + (double)(m->n[a] - 1) * m->spacing[a];
    }
    const double aim_z = (double)o->d.aim_z.hi + (double)o->d.aim_z.lo;
    const double aim_r = (double)o->d.aim_r.hi + (double)o->d.aim_r.lo;
    if (!(aim_z > hi[2])) return serr(PIVBOS_ERR_UNSUPPORTED, "the surrogate needs the lens after the density box");
    pivbos_surrogate* sg = new (std::nothrow) pivbos_surrogate();
    if (!sg) return serr(PIVBOS_ERR_OOM, "host allocation");
    sg->device = dev;
    sg->integrator = integrator;
    sg->medium = m;
    sg->medium_version = m->version;
    sg->optics = o;
    memset(&sg->rep, 0, sizeof sg->rep);
    pivbos_surrogate_report& R = sg->rep;
    pivbos::SurrParams& S = sg->S;
    memset(&S, 0, sizeof S);
    const double z_ref = std::isnan(c.ref_plane_z) ? 0.5 * (lo[2] + hi[2]) : c.ref_plane_z;
    S.z_lo = to_dfc2(lo[2]);
    S.z_ref = to_dfc2(z_ref);
    S.cx = (float)(0.5 * (lo[0] + hi[0]));
    S.cy = (float)(0.5 * (lo[1] + hi[1]));
    S.cz = (float)(0.5 * (lo[2] + hi[2]));
    S.hx = (float)(0.5 * (hi[0] - lo[0]));
    S.hy = (float)(0.5 * (hi[1] - lo[1]));
    S.hz = (float)fmax(0.5 * (hi[2] - lo[2]), 1e-9);
    S.u_scale = (float)((aim_r + fmax(fabs(S.cx) + S.hx, fabs(S.cy) + S.hy)) / (aim_z - hi[2]));
    S.inv_h[0] = 1.0f / S.hx;
    S.inv_h[1] = 1.0f / S.hy;
    S.inv_h[2] = 1.0f / S.hz;
    S.inv_u_scale = 1.0f / S.u_scale;
    for (int q = 0; q < 4; ++q) S.t_scale[q] = S.b_scale[q] = S.inv_b_scale[q] = 1.0f;
    S.nbx = 16;
    S.nby = 16;
    S.nbz = 16;
    S.nbu = 4;
    S.use_net = c.use_network == 1 ? 1 : 0;
    // -1: chosen below from the pilot rays; until then the table is built
    // and the pilot runs with a nonzero count
    S.born_k = c.born_segments < 0 ? 8 : c.born_segments;
    const int nbins = pivbos::kSurrBins;
    cudaError_t e = pivbos::mlp_alloc(sg->net, 128);
    if (e == cudaSuccess) e = cudaMalloc(&sg->bin_ok, sizeof(uint32_t) * (nbins / 32));
    if (e == cudaSuccess) e = cudaMalloc(&sg->bin_net, sizeof(uint32_t) * (nbins / 32));
    if (e != cudaSuccess) {
        pivbos_surrogate_destroy(sg);
        return scuda(e, "surrogate allocation");
    }
    // ---- projection table: columns through the pupil centre over the box's
    // back face, one level per grid node in depth
    const double t_start = now_s();
    if (S.born_k > 0) {
        const double persp = aim_z - hi[2];
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
        for (int cnr = 0; cnr < 8; ++cnr) {
            const double x = (cnr & 1) ? hi[0] : lo[0], y = (cnr & 2) ? hi[1] : lo[1], z = (cnr & 4) ? hi[2] : lo[2];
            const double f = persp / (aim_z - z);
            xmin = fmin(xmin, x * f); xmax = fmax(xmax, x * f);
            ymin = fmin(ymin, y * f); ymax = fmax(ymax, y * f);
        }
        const int lpc = c.table_levels_per_cell;
        S.tnz = std::max(2, std::min(lpc * (m->n[2] - 1) + 1, 1024));
        // columns per grid spacing: as configured, or the densest of 4, 2, 1
        // whose table fits in 16 GiB (lateral interpolation of the column
        // integrals is the projection's accuracy limit)
        int cpc = c.table_columns_per_cell;
        if (cpc == 0) {
            for (cpc = 4; cpc > 1; cpc /= 2) {
                const double cols = (double)std::min(cpc * (m->n[0] - 1) + 1, 2048) *
                                    (double)std::min(cpc * (m->n[1] - 1) + 1, 2048);
                if (cols * S.tnz * 2 * sizeof(float4) <= 16.0 * (1ull << 30)) break;
            }
        }
        S.tnx = std::min(cpc * (m->n[0] - 1) + 1, 2048);
        S.tny = std::min(cpc * (m->n[1] - 1) + 1, 2048);
        R.table_columns_per_cell = cpc;
        S.t_x0 = (float)xmin;
        S.t_y0 = (float)ymin;
        S.t_inv_dx = (float)((S.tnx - 1) / fmax(xmax - xmin, 1e-12));
        S.t_inv_dy = (float)((S.tny - 1) / fmax(ymax - ymin, 1e-12));
        S.t_inv_dz = (float)((S.tnz - 1) / fmax(hi[2] - lo[2], 1e-12));
        S.zlo_f = (float)lo[2];
        S.zhi_f = (float)hi[2];
        S.aim_z = (float)aim_z;
        S.persp = (float)persp;
        const size_t nodes = (size_t)S.tnx * S.tny * S.tnz;
        e = cudaMalloc(&sg->table, nodes * 2 * sizeof(float4));
        if (e == cudaSuccess) {
            const double level = (hi[2] - lo[2]) / (S.tnz - 1);
            const int sub = (int)std::min(64.0, std::max(2.0, ceil(4.0 * level / m->spacing[2])));
            const int cols = S.tnx * S.tny;
            pivbos::surr_table_kernel<<<(cols + 127) / 128, 128, 0, s>>>(P.m, S, sub, sg->table);
            pivbos::count_launches(1);
            e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) {
            pivbos_surrogate_destroy(sg);
            return scuda(e, "surrogate projection table");
        }
        S.table = sg->table;
        S.table_h = sg->table + nodes;
        R.table_bytes = (double)(nodes * 2 * sizeof(float4));
    }
    R.seconds_table = now_s() - t_start;
    // ---- S1: pilot statistics, then training and held-out samples traced
    // by the plain path
    const double t0 = now_s();
    DevBuf<__nv_bfloat16> Xt, Xv;
    DevBuf<float> Tt, Yv;
    DevBuf<uint64_t> idv;
    DevBuf<double> refpx, pilot, accd;
    DevBuf<int> refst;
    DevBuf<unsigned int> bincnt;
    // the training set is allocated when the network is trained
    e = Xv.alloc((size_t)c.n_val * pivbos::kMlpIn);
    if (e == cudaSuccess) e = Yv.alloc((size_t)c.n_val * 4);
    if (e == cudaSuccess) e = idv.alloc((size_t)c.n_val);
    if (e == cudaSuccess) e = refpx.alloc((size_t)c.n_val * 2);
    if (e == cudaSuccess) e = refst.alloc((size_t)c.n_val);
    if (e == cudaSuccess) e = pilot.alloc(18 + pivbos::kPilotK);
    if (e == cudaSuccess) e = accd.alloc((size_t)4 * nbins + 5);
    if (e == cudaSuccess) e = bincnt.alloc(nbins);
    if (e != cudaSuccess) {
        pivbos_surrogate_destroy(sg);
        return scuda(e, "surrogate data allocation");
    }
    const int64_t n_pilot = std::min<int64_t>(c.n_val, 65536);
    const int npv = 18 + pivbos::kPilotK;
    e = cudaMemsetAsync(pilot.p, 0, sizeof(double) * npv, s);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n_pilot + 127) / 128);
        if (integrator == PIVBOS_RK4)
            pivbos::surr_pilot_kernel<PIVBOS_RK4><<<blocks, 128, 0, s>>>(P, S, total, n_pilot, c.seed, 1e-6, 1e-6, pilot.p);
        else
            pivbos::surr_pilot_kernel<PIVBOS_EULER><<<blocks, 128, 0, s>>>(P, S, total, n_pilot, c.seed, 1e-6, 1e-6, pilot.p);
        pivbos::count_launches(1);
    }
    double pm[18 + pivbos::kPilotK];
    if (e == cudaSuccess) e = cudaMemcpyAsync(pm, pilot.p, sizeof pm, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        pivbos_surrogate_destroy(sg);
        return scuda(e, "surrogate pilot");
    }
    // Segment count: the smallest candidate whose projection alone keeps
    // the pilot's RMS sensor error within 80 % of the budget the held-out
    // estimate may use (the network corrects part of it and the confidence
    // map turns away what is left over), else the largest candidate.  Each
    // halving of the segments halves the render's table lookups.
    if (c.born_segments < 0) {
        const double nk = pm[17 + pivbos::kPilotK];
        const double goal = 0.8 * c.budget_margin * c.err_budget_px;
        int kc = pivbos::kPilotK - 1;
        for (int q = 0; q < pivbos::kPilotK; ++q)
            if (nk > 0 && sqrt(pm[17 + q] / nk) <= goal) {
                kc = q;
                break;
            }
        S.born_k = 1 << kc;
        if (kc != 3) {   // the pilot's moments used 8 segments: redo them with the chosen count
            e = cudaMemsetAsync(pilot.p, 0, sizeof(double) * npv, s);
            if (e == cudaSuccess) {
                const unsigned blocks = (unsigned)((n_pilot + 127) / 128);
                if (integrator == PIVBOS_RK4)
                    pivbos::surr_pilot_kernel<PIVBOS_RK4><<<blocks, 128, 0, s>>>(P, S, total, n_pilot, c.seed, 1e-6,
                                                                                1e-6, pilot.p);
                else
                    pivbos::surr_pilot_kernel<PIVBOS_EULER><<<blocks, 128, 0, s>>>(P, S, total, n_pilot, c.seed,
                                                                                  1e-6, 1e-6, pilot.p);
                pivbos::count_launches(1);
            }
            double keep[pivbos::kPilotK + 1];
            for (int q = 0; q <= pivbos::kPilotK; ++q) keep[q] = pm[17 + q];
            if (e == cudaSuccess) e = cudaMemcpyAsync(pm, pilot.p, sizeof pm, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (int q = 0; q <= pivbos::kPilotK; ++q) pm[17 + q] = keep[q];
            if (e != cudaSuccess) {
                pivbos_surrogate_destroy(sg);
                return scuda(e, "surrogate pilot");
            }
        }
    }
    R.born_segments = S.born_k;
    {
        const double nk = pm[17 + pivbos::kPilotK];
        for (int q = 0; q < pivbos::kPilotK; ++q) R.pilot_rms_px_born_k[q] = nk > 0 ? sqrt(pm[17 + q] / nk) : 0.0;
    }
    // Scales.  Network inputs: the projection residual per component at unit
    // RMS.  Network outputs: the correction in units of its RMS effect on
    // the sensor (J_q px per unit, measured about the straight rays), so the
    // loss weighs errors by what they move on the image, at about unit RMS
    // overall.
    double J[4], cc = 0.0;
    for (int q = 0; q < 4; ++q) {
        R.target_rms[q] = sqrt(pm[q] / n_pilot);
        const double brms = sqrt(pm[4 + q] / n_pilot);
        R.correction_rms[q] = sqrt(pm[8 + q] / n_pilot);
        S.b_scale[q] = (float)(brms > 1e-30 ? brms : 1.0);
        S.inv_b_scale[q] = 1.0f / S.b_scale[q];
        J[q] = pm[16] > 0 ? sqrt(pm[12 + q] / pm[16]) : 0.0;
        R.sensor_px_per_unit[q] = J[q];
        cc += (R.correction_rms[q] * J[q]) * (R.correction_rms[q] * J[q]) / 4.0;
    }
    cc = sqrt(cc);
    for (int q = 0; q < 4; ++q) {
        double scale = (J[q] > 0 && cc > 0) ? cc / J[q] : R.correction_rms[q];
        if (!(scale > 1e-30)) scale = 1e-30;
        S.t_scale[q] = (float)scale;
    }
    auto data = [&](int64_t n, uint32_t streamid, __nv_bfloat16* X, float* T, uint64_t* ids, double* rp, int* rs) {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        if (integrator == PIVBOS_RK4)
            pivbos::surr_data_kernel<PIVBOS_RK4><<<blocks, 128, 0, s>>>(P, S, total, n, streamid, c.seed, X, T, ids, rp, rs);
        else
            pivbos::surr_data_kernel<PIVBOS_EULER><<<blocks, 128, 0, s>>>(P, S, total, n, streamid, c.seed, X, T, ids, rp, rs);
        pivbos::count_launches(1);
    };
    data(c.n_val, 1, Xv.p, nullptr, idv.p, refpx.p, refst.p);
    e = cudaStreamSynchronize(s);
    R.seconds_data = now_s() - t0;
    // ---- S2: training on the GPU (its data first: plain-traced rays)
    auto train = [&]() -> cudaError_t {
        const double td = now_s();
        cudaError_t et = Xt.alloc((size_t)c.n_train * pivbos::kMlpIn);
        if (et == cudaSuccess) et = Tt.alloc((size_t)c.n_train * 4);
        if (et != cudaSuccess) return et;
        data(c.n_train, 0, Xt.p, Tt.p, nullptr, nullptr, nullptr);
        et = cudaStreamSynchronize(s);
        R.seconds_data += now_s() - td;
        if (et != cudaSuccess) return et;
        const double t1 = now_s();
        std::vector<float> p0;
        init_params(p0, c.seed);
        et = cudaMemcpy(sg->net.params, p0.data(), sizeof(float) * p0.size(), cudaMemcpyHostToDevice);
        if (et == cudaSuccess) et = pivbos::mlp_sync_bf16(sg->net, s);
        pivbos::MlpWork w;
        if (et == cudaSuccess) et = pivbos::mlp_work_alloc(w, c.batch);
        const int64_t per_epoch = (c.n_train + c.batch - 1) / c.batch;
        const int64_t steps = per_epoch * c.epochs;
        double last_loss = 0.0;
        for (int64_t t = 0; t < steps && et == cudaSuccess; ++t) {
            const int64_t off = (t % per_epoch) * c.batch;
            const int rows = (int)std::min<int64_t>(c.batch, c.n_train - off);
            const float lr = (float)(c.lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(M_PI * (double)t / (double)steps))));
            et = pivbos::mlp_forward(sg->net, Xt.p + off * pivbos::kMlpIn, rows, w.y, &w, Tt.p + off * 4, s);
            if (et == cudaSuccess) et = pivbos::mlp_backward(sg->net, Xt.p + off * pivbos::kMlpIn, rows, w, s);
            if (et == cudaSuccess) et = pivbos::mlp_adam(sg->net, (int)(t + 1), lr, s);
            if (et == cudaSuccess && t == steps - 1) {
                double l = 0.0;
                et = cudaMemcpyAsync(&l, w.loss, sizeof l, cudaMemcpyDeviceToHost, s);
                if (et == cudaSuccess) et = cudaStreamSynchronize(s);
                last_loss = l / ((double)rows * pivbos::kMlpOut);
            }
        }
        pivbos::mlp_work_free(w);
        R.train_loss = last_loss;
        R.train_steps = (double)steps;
        R.network_trained = 1.0;
        R.seconds_train += now_s() - t1;
        return et;
    };
    // ---- confidence map: the plain tracer judges the predictors on the
    // held-out rays, per bin (with_net: the network's outputs, else zero)
    const size_t nacc = (size_t)4 * nbins + 5;
    std::vector<double> hd(nacc);
    std::vector<unsigned int> hc(nbins);
    auto evaluate = [&](bool with_net) -> cudaError_t {
        const double t2 = now_s();
        cudaError_t ev = with_net ? pivbos::mlp_forward(sg->net, Xv.p, (int)c.n_val, Yv.p, nullptr, nullptr, s)
                                  : cudaMemsetAsync(Yv.p, 0, sizeof(float) * 4 * (size_t)c.n_val, s);
        if (ev == cudaSuccess) ev = cudaMemsetAsync(accd.p, 0, sizeof(double) * nacc, s);
        if (ev == cudaSuccess) ev = cudaMemsetAsync(bincnt.p, 0, sizeof(unsigned int) * nbins, s);
        if (ev == cudaSuccess) {
            pivbos::BinAcc acc{{accd.p, accd.p + nbins, accd.p + 2 * (size_t)nbins}, accd.p + 3 * (size_t)nbins,
                               bincnt.p, accd.p + 4 * (size_t)nbins};
            pivbos::surr_eval_kernel<<<(unsigned)((c.n_val + 127) / 128), 128, 0, s>>>(P, S, idv.p, Yv.p, refpx.p,
                                                                                       refst.p, c.n_val, acc);
            pivbos::count_launches(1);
        }
        if (ev == cudaSuccess)
            ev = cudaMemcpyAsync(hd.data(), accd.p, sizeof(double) * nacc, cudaMemcpyDeviceToHost, s);
        if (ev == cudaSuccess)
            ev = cudaMemcpyAsync(hc.data(), bincnt.p, sizeof(unsigned) * nbins, cudaMemcpyDeviceToHost, s);
        if (ev == cudaSuccess) ev = cudaStreamSynchronize(s);
        R.seconds_validate += now_s() - t2;
        return ev;
    };
    if (e == cudaSuccess) e = c.use_network == 1 ? train() : cudaSuccess;
    if (e == cudaSuccess) e = evaluate(c.use_network == 1);
    if (e != cudaSuccess) {
        pivbos_surrogate_destroy(sg);
        return scuda(e, "surrogate training");
    }
    auto sums = [&](std::vector<double>* err2, std::vector<double>& stp, double* tot, double* all_err,
                    double& all_steps) {
        for (int v = 0; v < 3; ++v)
            err2[v].assign(hd.begin() + (size_t)v * nbins, hd.begin() + (size_t)(v + 1) * nbins);
        stp.assign(hd.begin() + 3 * (size_t)nbins, hd.begin() + 4 * (size_t)nbins);
        for (int q = 0; q < 5; ++q) tot[q] = hd[4 * (size_t)nbins + q];
        all_steps = 0.0;
        for (int v = 0; v < 3; ++v) all_err[v] = 0.0;
        for (int b = 0; b < nbins; ++b) {
            for (int v = 0; v < 3; ++v) all_err[v] += err2[v][b];
            all_steps += stp[b];
        }
    };
    std::vector<double> err2[3], stp;
    double tot[5], all_err[3], all_steps = 0.0;
    sums(err2, stp, tot, all_err, all_steps);
    const double margin = c.budget_margin;
    const double budget2 = margin * margin * (double)c.err_budget_px * c.err_budget_px * tot[0];
    const double n_reached = tot[0], n_box = tot[1];
    // Automatic mode: the network is trained only when the projection alone,
    // served within the budget, would leave more than 1 % of the plain
    // path's integration work to the fallback; the projection alone then
    // serves and no network runs.
    bool mixed = false;
    if (c.use_network == -1) {
        const Served pv = choose_bins(err2[1], stp, hc, c.min_bin_count, budget2, nullptr);
        if (all_steps > 0 && pv.steps < kAutoTrainBelow * all_steps) {
            e = train();
            if (e == cudaSuccess) e = evaluate(true);
            if (e != cudaSuccess) {
                pivbos_surrogate_destroy(sg);
                return scuda(e, "surrogate training");
            }
            sums(err2, stp, tot, all_err, all_steps);
            mixed = true;
        }
    }
    std::vector<uint32_t> ok(nbins / 32, 0u), netb(nbins / 32, 0u);
    auto rms = [&](double e2, double flips) { return n_box > flips ? sqrt(e2 / (n_box - flips)) : 0.0; };
    Served sv[3];
    if (mixed) {
        // per bin: the projection alone, the projection with the network's
        // correction, or the plain fallback, whichever costs least under the
        // error budget
        Mixed mx = choose_mixed(err2[0], err2[1], stp, hc, c.min_bin_count, budget2, S.born_k, true, &ok, &netb);
        // the plan without the network, rendered by the direct pass, when
        // it costs less than the plan with it on the list-based kernels
        if (mx.net_rays > 0) {
            std::vector<uint32_t> ok_p(nbins / 32, 0u), net_p(nbins / 32, 0u);
            const Mixed mp =
                choose_mixed(err2[0], err2[1], stp, hc, c.min_bin_count, budget2, S.born_k, false, &ok_p, &net_p);
            if (mp.cost - kCostListRay * mp.rays <= mx.cost) {
                mx = mp;
                ok = ok_p;
                netb = net_p;
            }
        }
        sv[0] = choose_bins(err2[0], stp, hc, c.min_bin_count, budget2, nullptr);
        sv[1] = choose_bins(err2[1], stp, hc, c.min_bin_count, budget2, nullptr);
        sv[2] = choose_bins(err2[2], stp, hc, c.min_bin_count, budget2, nullptr);
        double e_pred = 0.0;
        for (int b = 0; b < nbins; ++b) e_pred += ((netb[b >> 5] >> (b & 31)) & 1u) ? err2[0][b] : err2[1][b];
        S.use_net = mx.net_rays > 0 ? 2 : 0;
        R.val_rms_px = rms(e_pred, tot[3]);
        R.val_rms_px_served = n_reached > 0 ? sqrt(mx.err2 / n_reached) : 0.0;
        R.val_served_frac = n_box > 0 ? mx.rays / n_box : 0.0;
        R.val_served_frac_net = n_box > 0 ? mx.net_rays / n_box : 0.0;
        R.steps_saved_frac = all_steps > 0 ? mx.steps / all_steps : 0.0;
        R.val_status_flip_frac = n_box > 0 ? tot[3] / n_box : 0.0;
    } else {
        // one predictor for every served bin: the network's (forced), or the
        // projection alone
        const int vs = c.use_network == 1 ? 0 : 1;
        for (int v = 0; v < 3; ++v)
            sv[v] = choose_bins(err2[v], stp, hc, c.min_bin_count, budget2, v == vs ? &ok : nullptr);
        S.use_net = c.use_network == 1 ? 1 : 0;
        R.val_rms_px = rms(all_err[vs], tot[2 + vs]);
        R.val_rms_px_served = n_reached > 0 ? sqrt(sv[vs].err2 / n_reached) : 0.0;
        R.val_served_frac = n_box > 0 ? sv[vs].rays / n_box : 0.0;
        R.val_served_frac_net = vs == 0 ? R.val_served_frac : 0.0;
        R.steps_saved_frac = all_steps > 0 ? sv[vs].steps / all_steps : 0.0;
        R.val_status_flip_frac = n_box > 0 ? tot[2 + vs] / n_box : 0.0;
    }
    R.val_rms_px_born = rms(all_err[1], tot[3]);
    R.val_rms_px_straight = rms(all_err[2], tot[4]);
    R.val_served_frac_born = n_box > 0 ? sv[1].rays / n_box : 0.0;
    R.val_served_frac_straight = n_box > 0 ? sv[2].rays / n_box : 0.0;
    R.steps_saved_frac_born = all_steps > 0 ? sv[1].steps / all_steps : 0.0;
    R.steps_saved_frac_straight = all_steps > 0 ? sv[2].steps / all_steps : 0.0;
    R.n_val_reached = n_reached;
    R.n_val_box = n_box;
    e = cudaMemcpy(sg->bin_ok, ok.data(), sizeof(uint32_t) * ok.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sg->bin_net, netb.data(), sizeof(uint32_t) * netb.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pivbos_surrogate_destroy(sg);
        return scuda(e, "surrogate bins");
    }
    S.bin_ok = sg->bin_ok;
    S.bin_net = sg->bin_net;
    if (report) *report = R;
    *out = sg;
    return PIVBOS_OK;
}

static pivbos_status surr_prepare(const pivbos_surrogate* sg, const pivbos_frame_desc* frame, pivbos::TraceParams& P,
                                  uint64_t& total)
{
    if (!sg || !frame) return serr(PIVBOS_ERR_INVALID_ARG, "surrogate and frame are required");
    if (frame->medium != sg->medium || frame->optics != sg->optics)
        return serr(PIVBOS_ERR_INVALID_ARG, "the frame must use the medium and optics the surrogate was trained on");
    if (sg->medium->version != sg->medium_version)
        return serr(PIVBOS_ERR_INVALID_ARG, "the medium was refilled after the surrogate was trained");
    int dev = 0;
    pivbos_status st = pivbos::prepare_trace(frame->medium, frame->optics, frame->sources, frame->n_sources, 1,
                                             frame->rays_per_source, frame->seed, frame->frame, sg->integrator,
                                             frame->step, &P, &dev, &total);
    if (st) return st;
    if (dev != sg->device) return serr(PIVBOS_ERR_INVALID_ARG, "surrogate belongs to device %d", sg->device);
    return PIVBOS_OK;
}

static pivbos_status surrogate_render_impl(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                           int64_t first_source, int64_t* n_fallback, void* stream);

pivbos_status pivbos_surrogate_render(const pivbos_surrogate* sg, const pivbos_frame_desc* frame, int64_t* n_fallback,
                                      void* stream)
{
    return surrogate_render_impl(sg, frame, 0, n_fallback, stream);
}

pivbos_status pivbos_surrogate_render_range(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                            int64_t first_source, int64_t* n_fallback, void* stream)
{
    pivbos::set_last_error("");
    if (!frame) return serr(PIVBOS_ERR_INVALID_ARG, "frame is NULL");
    if (first_source < 0 || frame->n_sources < 0 || first_source + frame->n_sources > 0xffffffffll)
        return serr(PIVBOS_ERR_INVALID_ARG, "first_source %lld outside [0, 2^32 - n_sources]", (long long)first_source);
    return surrogate_render_impl(sg, frame, first_source, n_fallback, stream);
}

static pivbos_status surrogate_render_impl(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                           int64_t first_source, int64_t* n_fallback, void* stream)
{
    pivbos::set_last_error("");
    pivbos::TraceParams P;
    uint64_t total = 0;
    pivbos_status st = surr_prepare(sg, frame, P, total);
    if (st) return st;
    P.source_offset = (uint32_t)first_source;
    cudaPointerAttributes a;
    if (!frame->image || cudaPointerGetAttributes(&a, frame->image) != cudaSuccess ||
        a.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return serr(PIVBOS_ERR_INVALID_ARG, "image must be device memory");
    }
    if (n_fallback) *n_fallback = 0;
    if (total == 0) return PIVBOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)frame->n_sources;
    uint32_t n_pow2 = 2;
    while (n_pow2 < n) n_pow2 <<= 1;
    const uint32_t capacity = (uint32_t)total;
    const size_t off_perm = (size_t)n_pow2 * 8;
    const size_t off_sdf = off_perm + (((size_t)n * 4 + 255) & ~(size_t)255);
    const size_t off_cnt = off_sdf + (((size_t)n * 24 + 255) & ~(size_t)255);
    const size_t off_fb = off_cnt + 256;
    const size_t bytes = off_fb + (size_t)capacity * 4;
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, bytes, s);
    if (e != cudaSuccess) return scuda(e, "surrogate render scratch");
    uint32_t* perm = (uint32_t*)(scratch + off_perm);
    float2* sdf = (float2*)(scratch + off_sdf);
    // [0] render items, [1] fallback rays, [2] fallback chunks
    unsigned long long* counters = (unsigned long long*)(scratch + off_cnt);
    uint32_t* fb = (uint32_t*)(scratch + off_fb);
    e = pivbos::launch_morton_sort(frame->sources, n, (uint64_t*)scratch, n_pow2, perm, sdf, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), s);
    P.perm = perm;
    P.src_df = sdf;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sg->device);
    // no bin takes the network: one direct pass (no served list), unless
    // PIVBOS_SURR_DIRECT=0 asks for the three-kernel path (read per call, so
    // that a check can render both ways)
    const char* dir_env = getenv("PIVBOS_SURR_DIRECT");
    const bool direct = sg->S.use_net == 0 && !(dir_env && atoi(dir_env) == 0);
    if (e == cudaSuccess && direct) {
        const uint64_t items = (total + pivbos::kMaxOrderRays - 1) / pivbos::kMaxOrderRays;
        const unsigned grid = (unsigned)std::min<uint64_t>(items, (uint64_t)sms * pivbos::kDirectCtasPerSm);
        pivbos::timing_begin("surrogate_direct", s);
        if (pivbos::optics_ext(P.o))
            pivbos::surr_direct_kernel<true><<<grid, 256, 0, s>>>(P, sg->S, 0, total, fb, counters + 1, capacity,
                                                                  frame->image, frame->stats);
        else
            pivbos::surr_direct_kernel<false><<<grid, 256, 0, s>>>(P, sg->S, 0, total, fb, counters + 1, capacity,
                                                                   frame->image, frame->stats);
        pivbos::timing_end("surrogate_direct", s);
        pivbos::count_launches(1);
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        // three kernels per chunk of up to 2^26 rays: prep -> network -> finish
        const uint64_t chunk = std::min<uint64_t>(total, 1ull << 26);
        const int use_net = sg->S.use_net;
        pivbos::ServedList sv;
        memset(&sv, 0, sizeof sv);
        char* sbuf = nullptr;
        // per entry: network input 32 B, projection residual 16 B, full
        // residual 16 B, straight line 16 B, ray id 4 B, network slot 4 B
        const size_t off_count = ((size_t)chunk * 88 + 255) & ~(size_t)255;
        const size_t sbytes = off_count + 256;
        e = cudaMallocAsync((void**)&sbuf, sbytes, s);
        if (e == cudaSuccess) {
            sv.X = (__nv_bfloat16*)sbuf;
            sv.B = (float4*)(sbuf + (size_t)chunk * 32);
            sv.R = (float4*)(sbuf + (size_t)chunk * 48);
            sv.L = (float4*)(sbuf + (size_t)chunk * 64);
            sv.ids = (uint32_t*)(sbuf + (size_t)chunk * 80);
            // [0] served, [1] finish items, [2] network rays
            sv.count = (unsigned long long*)(sbuf + off_count);
            sv.capacity = (uint32_t)chunk;
            if (use_net == 2) {
                sv.net_idx = (uint32_t*)(sbuf + (size_t)chunk * 84);
                sv.net_count = sv.count + 2;
            }
            for (uint64_t c0 = 0; c0 < total && e == cudaSuccess; c0 += chunk) {
                const uint64_t c1 = std::min(total, c0 + chunk);
                e = cudaMemsetAsync(sv.count, 0, 3 * sizeof(unsigned long long), s);
                if (e != cudaSuccess) break;
                const uint64_t items = (c1 - c0 + pivbos::kMaxOrderRays - 1) / pivbos::kMaxOrderRays;
                pivbos::timing_begin("surrogate_prep", s);
                pivbos::surr_prep_kernel<<<(unsigned)std::min<uint64_t>(items, (uint64_t)sms * 6), 256, 0, s>>>(
                    P, sg->S, c0, c1, sv, fb, counters + 1, capacity);
                pivbos::timing_end("surrogate_prep", s);
                pivbos::count_launches(1);
                if (use_net) {
                    e = pivbos::launch_surr_net(sg->S, sg->net.wbf, sg->net.params, sv, P.status_word, s);
                    if (e != cudaSuccess) break;
                }
                pivbos::timing_begin("surrogate_finish", s);
                if (pivbos::optics_ext(P.o))
                    pivbos::surr_finish_kernel<true><<<sms * pivbos::kFinishCtasPerSm, 256, 0, s>>>(
                        P, sg->S, sv, use_net ? sv.R : sv.B, frame->image, frame->stats, sv.count + 1);
                else
                    pivbos::surr_finish_kernel<false><<<sms * pivbos::kFinishCtasPerSm, 256, 0, s>>>(
                        P, sg->S, sv, use_net ? sv.R : sv.B, frame->image, frame->stats, sv.count + 1);
                pivbos::timing_end("surrogate_finish", s);
                pivbos::count_launches(1);
                e = cudaGetLastError();
            }

            cudaError_t ef = cudaFreeAsync(sbuf, s);
            if (e == cudaSuccess) e = ef;
        }
    }
    if (e == cudaSuccess) {
        pivbos::TraceParams PL = P;
        PL.ray_list = fb;
        pivbos::timing_begin("surrogate_fallback", s);
        e = pivbos::launch_list(PL, sg->integrator, counters + 1, capacity, frame->image, frame->stats, 2048u,
                                counters + 2, s);
        pivbos::timing_end("surrogate_fallback", s);
    }
    unsigned long long nfb = 0;
    if (e == cudaSuccess && n_fallback) {
        e = cudaMemcpyAsync(&nfb, counters + 1, sizeof nfb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        *n_fallback = (int64_t)nfb;
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return scuda(e, "surrogate render");
    if (ef != cudaSuccess) return scuda(ef, "surrogate render scratch release");
    return PIVBOS_OK;
}

pivbos_status pivbos_surrogate_sensor(const pivbos_surrogate* sg, const pivbos_frame_desc* frame,
                                      const int64_t* ray_ids, int64_t n, double* sensor_xy, int32_t* flags,
                                      int32_t* status, void* stream)
{
    pivbos::set_last_error("");
    pivbos::TraceParams P;
    uint64_t total = 0;
    pivbos_status st = surr_prepare(sg, frame, P, total);
    if (st) return st;
    if (n < 0 || n > (1ll << 31) || (n > 0 && (!ray_ids || !sensor_xy || !flags || !status)))
        return serr(PIVBOS_ERR_INVALID_ARG, "ray ids and outputs are required");
    if (n == 0) return PIVBOS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf<__nv_bfloat16> X;
    DevBuf<float> Y;
    cudaError_t e = X.alloc((size_t)n * pivbos::kMlpIn);
    if (e == cudaSuccess) e = Y.alloc((size_t)n * 4);
    if (e != cudaSuccess) return scuda(e, "surrogate sensor scratch");
    const unsigned blocks = (unsigned)((n + 127) / 128);
    if (sg->S.use_net) {
        pivbos::surr_features_kernel<<<blocks, 128, 0, s>>>(P, sg->S, ray_ids, n, X.p);
        pivbos::count_launches(1);
        e = pivbos::mlp_forward(sg->net, X.p, (int)n, Y.p, nullptr, nullptr, s);
    } else {
        e = cudaMemsetAsync(Y.p, 0, sizeof(float) * 4 * (size_t)n, s);
    }
    if (e == cudaSuccess) {
        if (sg->integrator == PIVBOS_RK4)
            pivbos::surr_sensor_kernel<PIVBOS_RK4><<<blocks, 128, 0, s>>>(P, sg->S, Y.p, ray_ids, n, sensor_xy, flags,
                                                                         status);
        else
            pivbos::surr_sensor_kernel<PIVBOS_EULER><<<blocks, 128, 0, s>>>(P, sg->S, Y.p, ray_ids, n, sensor_xy,
                                                                           flags, status);
        pivbos::count_launches(1);
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return scuda(e, "surrogate sensor");
    return PIVBOS_OK;
}

pivbos_status pivbos_surrogate_report_get(const pivbos_surrogate* sg, pivbos_surrogate_report* out)
{
    if (!sg || !out) return serr(PIVBOS_ERR_INVALID_ARG, "NULL argument");
    *out = sg->rep;
    return PIVBOS_OK;
}

void pivbos_surrogate_destroy(pivbos_surrogate* sg)
{
    if (!sg) return;
    pivbos::mlp_free(sg->net);
    cudaFree(sg->bin_ok);
    cudaFree(sg->bin_net);
    cudaFree(sg->table);
    delete sg;
}

}  // extern "C"
