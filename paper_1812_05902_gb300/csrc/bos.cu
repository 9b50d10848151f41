// The simulated BOS experiment of Sec. 4: per-dot light-ray displacements
// (each ray traced through the medium and, with the same lens point,
// through the uniform medium), the theoretical displacement of Eq. 9 along
// each dot's chief ray, and the bilinear map onto a regular grid the paper
// draws both on.
//
// Determinism: the per-dot sums and the grid sums are integers (fixed point),
// so atomics in any order give the same bits run to run.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "handles.cuh"
#include "trace.cuh"

namespace pivbos {

constexpr int kBosThreads = 256;
constexpr int kBosFields = 5;          // per dot: pairs, sum x0, sum y0, sum dx, sum dy
constexpr float kQ24 = 16777216.0f;    // the per-dot sums count 2^-24 px

// round(x * 2^24) for a double-float x with |x| < 2^26 px, with FP32/INT32
// instructions only (a 64-bit float-to-integer conversion would run on the
// FP64 pipe).  h = hi * 2^24 is exact; a = rint(h) and h - a are exact; the
// rest of the rounding comes from the low part.
__device__ __forceinline__ long long q24(df x)
{
    const float h = x.hi * kQ24;
    const float a = rintf(h);
    const float b = rintf((h - a) + x.lo * kQ24);
    const float ah = truncf(a * 0x1p-20f);
    const float al = a - ah * 0x1p20f;
    return (long long)(int)ah * (1ll << 20) + (long long)(int)al + (long long)(int)b;
}

// Work: like the render, the flattened (Morton slot, ray) space is cut into
// chunks of rays_per_cta consecutive rays, one chunk per CTA, traced in
// mid-plane Morton order in dense media (order_chunk), so that a warp's field
// gathers hit few cells.  A ray counts when it reaches the sensor both
// through the medium and through the uniform medium.  Sums go to per-slot
// accumulators: a warp reduces its rays slot by slot (the rays of a chunk
// belong to few slots), the lane holding a slot's sum adds it to the CTA's
// shared accumulators (the first kBosSharedSlots slots of the chunk) or, past
// them, to the global ones; the CTA then adds its shared sums to the global
// accumulators.  All sums are integers, so the order does not matter.
constexpr int kBosSharedSlots = 32;

struct BosShared {
    uint32_t order[kMaxOrderRays];
    unsigned long long acc[kBosSharedSlots * kBosFields];
};

template <int INTEG, bool CACHE, bool EXT>
__global__ void __launch_bounds__(kBosThreads, CACHE ? 2 : 3)
bos_pairs_kernel(const TraceParams P, unsigned long long* __restrict__ acc, uint32_t rays_per_cta, uint64_t total)
{
    __shared__ BosShared sh;
    const uint64_t first = (uint64_t)blockIdx.x * rays_per_cta;
    const uint64_t last = min(first + rays_per_cta, total);
    const uint32_t n_here = (uint32_t)(last - first);
    const uint32_t rps = P.rays_per_source;
    const uint32_t slot0 = (uint32_t)(first / rps);
    for (int q = threadIdx.x; q < kBosSharedSlots * kBosFields; q += blockDim.x) sh.acc[q] = 0ull;
    const bool reorder = P.reorder && n_here <= (uint32_t)kMaxOrderRays;
    if (reorder) order_chunk(P, sh.order, first, n_here);   // ends with a barrier
    else __syncthreads();
    const int lane = threadIdx.x & 31;
    const int rounds = (int)((n_here + blockDim.x - 1) / blockDim.x);
    for (int round = 0; round < rounds; ++round) {
        const uint32_t e = (uint32_t)round * blockDim.x + threadIdx.x;
        const bool active = e < n_here;
        uint32_t slot = 0;
        long long v[kBosFields] = {0, 0, 0, 0, 0};
        if (active) {
            const uint64_t flat = first + (reorder ? (sh.order[e] & 0x7ffu) : e);
            slot = (uint32_t)(flat / rps);
            const uint32_t k = (uint32_t)(flat - (uint64_t)slot * rps);
            const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
            const float2* sp = P.src_df + 3 * (size_t)slot;
            const float2 a = __ldg(sp), b = __ldg(sp + 1), c = __ldg(sp + 2);
            const df sx = df{a.x, a.y}, sy = df{b.x, b.y}, sz = df{c.x, c.y};
            // the ray without the medium first (straight to the lens): only
            // its sensor position stays live across the traced ray
            df qx, qy;
            int st0 = PIVBOS_RAY_REACHED;
            {
                df dx, dy, dz;
                ray_start(P, sx, sy, sz, sid, k, dx, dy, dz);
                df Rx = sx, Ry = sy, Rz = sz;
                optics_to_sensor<DfOps, EXT>(P.o, Rx, Ry, Rz, dx, dy, dz, st0, qx, qy);
            }
            // the same ray (same lens point) through the medium
            RayOut r;
            trace_ray<INTEG, CACHE, EXT>(P, sx, sy, sz, sid, k, r, nullptr);
            if (r.status == PIVBOS_RAY_REACHED && st0 == PIVBOS_RAY_REACHED) {
                v[0] = 1;
                v[1] = q24(qx);
                v[2] = q24(qy);
                v[3] = q24(df_sub(r.px, qx));
                v[4] = q24(df_sub(r.py, qy));
            }
        }
        // the warp's pairs, one slot at a time
        const bool has = active && v[0] != 0;
        unsigned pending = __ballot_sync(0xffffffffu, has);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const uint32_t s_lead = __shfl_sync(0xffffffffu, slot, leader);
            const bool mine = has && slot == s_lead;
            const uint32_t ls = s_lead - slot0;
            unsigned long long* dst = ls < (uint32_t)kBosSharedSlots ? sh.acc + ls * kBosFields
                                                                     : acc + (size_t)kBosFields * s_lead;
#pragma unroll
            for (int q = 0; q < kBosFields; ++q) {
                long long w = mine ? v[q] : 0;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
                if (lane == leader && w != 0) atomicAdd(dst + q, (unsigned long long)w);
            }
            pending &= ~__ballot_sync(0xffffffffu, mine);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kBosSharedSlots * kBosFields; q += blockDim.x) {
        const unsigned long long x = sh.acc[q];
        if (x != 0ull) atomicAdd(acc + (size_t)kBosFields * slot0 + q, x);
    }
}

// Per-dot results from the per-slot sums (slot = position in Morton order,
// perm[slot] = the dot).
__global__ void bos_finish_kernel(const unsigned long long* __restrict__ acc, const uint32_t* __restrict__ perm,
                                  int64_t n, double* __restrict__ centroid, double* __restrict__ disp,
                                  int32_t* __restrict__ n_pairs)
{
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n) return;
    const unsigned long long* a = acc + (size_t)kBosFields * slot;
    const int64_t q = perm[slot];
    const long long c = (long long)a[0];
    if (n_pairs) n_pairs[q] = (int32_t)c;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double sc = c ? 0x1p-24 / (double)c : nan;
    if (centroid) {
        centroid[2 * q] = c ? (double)(long long)a[1] * sc : nan;
        centroid[2 * q + 1] = c ? (double)(long long)a[2] * sc : nan;
    }
    if (disp) {
        disp[2 * q] = c ? (double)(long long)a[3] * sc : nan;
        disp[2 * q + 1] = c ? (double)(long long)a[4] * sc : nan;
    }
}

// ---------------------------------------------------------------------------
// Eq. 9 along each dot's chief ray.  FP64 throughout: one thread per dot and
// a few samples per grid cell crossed, negligible next to tracing the dot's
// rays.
// ---------------------------------------------------------------------------
struct Eq9Geom {
    const float4* field;
    int n[3];
    double origin[3], h[3];
    double aim_z;
    double scale;     // M / (n0 * pitch): pixels per unit of Z_D * integral
    double z_mid;     // mid-plane of the box
};

// (dn/dx, dn/dy) sampled trilinearly at a point of the box (clamped)
__device__ __forceinline__ void sample_grad_xy(const Eq9Geom& G, double x, double y, double z, double& gx,
                                               double& gy)
{
    const double u[3] = {(x - G.origin[0]) / G.h[0], (y - G.origin[1]) / G.h[1], (z - G.origin[2]) / G.h[2]};
    int c[3];
    double f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = fmin(fmax(u[a], 0.0), (double)(G.n[a] - 1));
        c[a] = min((int)t, G.n[a] - 2);
        f[a] = t - (double)c[a];
    }
    const int sy = G.n[0], sz = G.n[0] * G.n[1];
    const float4* p = G.field + ((size_t)c[2] * G.n[1] + c[1]) * G.n[0] + c[0];
    gx = 0.0;
    gy = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int di = q & 1, dj = (q >> 1) & 1, dk = q >> 2;
        const double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        const float4 v = __ldg(p + dk * sz + dj * sy + di);
        gx += w * (double)v.y;
        gy += w * (double)v.z;
    }
}

// z where the line (x = s_ax + a (z - s_z)) crosses node plane i of axis
// `ax`; +inf past the last plane.
__device__ __forceinline__ double next_plane(const Eq9Geom& G, int ax, double s_ax, double s_z, double a, int i)
{
    if (i < 0 || i >= G.n[ax]) return INFINITY;
    return s_z + (G.origin[ax] + (double)i * G.h[ax] - s_ax) / a;
}

__global__ void __launch_bounds__(128)
bos_theory_kernel(const Eq9Geom G, const double* __restrict__ dots, int64_t n, double* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double s[3] = {dots[3 * q], dots[3 * q + 1], dots[3 * q + 2]};
    double Ix = 0.0, Iy = 0.0;
    if (G.aim_z != s[2]) {
        // the chief ray toward the lens centre (0, 0, aim_z), by z
        const double a[3] = {(0.0 - s[0]) / (G.aim_z - s[2]), (0.0 - s[1]) / (G.aim_z - s[2]), 1.0};
        double z0 = fmin(s[2], G.aim_z), z1 = fmax(s[2], G.aim_z);
        bool hit = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const double lo = G.origin[ax], hi = G.origin[ax] + (double)(G.n[ax] - 1) * G.h[ax];
            if (a[ax] == 0.0) {
                if (s[ax] < lo || s[ax] > hi) hit = false;
                continue;
            }
            const double za = s[2] + (lo - s[ax]) / a[ax];
            const double zb = s[2] + (hi - s[ax]) / a[ax];
            z0 = fmax(z0, fmin(za, zb));
            z1 = fmin(z1, fmax(za, zb));
        }
        if (hit && z1 > z0) {
            // walk the pieces between node-plane crossings in z order; the
            // sample is cubic in z on each, which two-point Gauss-Legendre
            // integrates exactly
            int idx[3], dir[3];
            double zn[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (a[ax] == 0.0) {
                    idx[ax] = -1;
                    dir[ax] = 0;
                    zn[ax] = INFINITY;
                    continue;
                }
                const double x0 = s[ax] + a[ax] * (z0 - s[2]);
                const double u = (x0 - G.origin[ax]) / G.h[ax];
                dir[ax] = a[ax] > 0.0 ? 1 : -1;
                idx[ax] = a[ax] > 0.0 ? (int)floor(u) + 1 : (int)ceil(u) - 1;
                zn[ax] = next_plane(G, ax, s[ax], s[2], a[ax], idx[ax]);
                for (int guard = 0; zn[ax] <= z0 && guard < 4; ++guard) {
                    idx[ax] += dir[ax];
                    zn[ax] = next_plane(G, ax, s[ax], s[2], a[ax], idx[ax]);
                }
            }
            const double g = 0.57735026918962576451;   // 1/sqrt(3)
            double zc = z0;
            const int max_pieces = G.n[0] + G.n[1] + G.n[2] + 4;
            for (int it = 0; it < max_pieces && zc < z1; ++it) {
                const double ze = fmin(z1, fmin(zn[0], fmin(zn[1], zn[2])));
                if (ze > zc) {
                    const double mid = 0.5 * (zc + ze), half = 0.5 * (ze - zc);
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const double z = t ? mid + half * g : mid - half * g;
                        double gx, gy;
                        sample_grad_xy(G, s[0] + a[0] * (z - s[2]), s[1] + a[1] * (z - s[2]), z, gx, gy);
                        Ix += half * gx;
                        Iy += half * gy;
                    }
                }
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (dir[ax] != 0 && zn[ax] <= ze) {
                        idx[ax] += dir[ax];
                        zn[ax] = next_plane(G, ax, s[ax], s[2], a[ax], idx[ax]);
                    }
                }
                zc = ze;
            }
        }
    }
    const double f = G.scale * (G.z_mid - s[2]);
    out[2 * q] = f * Ix;
    out[2 * q + 1] = f * Iy;
}

// ---------------------------------------------------------------------------
// Bilinear map of scattered values onto a regular grid: every point gives
// the four nodes of its cell its value with bilinear weights; a node holds
// the weighted mean.  The weights are summed as multiples of 2^-40 and the
// weighted values as multiples of 2^-32 px.
// ---------------------------------------------------------------------------
constexpr double kRegridMaxValue = 256.0;    // |value| per component, px

__global__ void regrid_splat_kernel(const double* __restrict__ xy, const double* __restrict__ vals, int64_t n,
                                    int W, int H, double x0, double y0, double inv_cell,
                                    unsigned long long* __restrict__ acc, int* __restrict__ status_word)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double x = xy[2 * q], y = xy[2 * q + 1], vx = vals[2 * q], vy = vals[2 * q + 1];
    if (!(isfinite(x) && isfinite(y) && isfinite(vx) && isfinite(vy))) return;
    const double u = (x - x0) * inv_cell, t = (y - y0) * inv_cell;
    if (!(u >= 0.0 && u <= (double)(W - 1) && t >= 0.0 && t <= (double)(H - 1))) return;
    if (fabs(vx) >= kRegridMaxValue || fabs(vy) >= kRegridMaxValue) {
        atomicCAS(status_word, 0, (int)PIVBOS_ERR_OVERFLOW);
        return;
    }
    const int i = min((int)u, W - 2), j = min((int)t, H - 2);
    const double fu = u - (double)i, fv = t - (double)j;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int di = c & 1, dj = c >> 1;
        const double w = (di ? fu : 1.0 - fu) * (dj ? fv : 1.0 - fv);
        unsigned long long* a = acc + 3 * ((size_t)(j + dj) * W + (i + di));
        const long long qw = __double2ll_rn(w * 0x1p40);
        if (qw == 0) continue;
        atomicAdd(a, (unsigned long long)qw);
        atomicAdd(a + 1, (unsigned long long)__double2ll_rn(w * vx * 0x1p32));
        atomicAdd(a + 2, (unsigned long long)__double2ll_rn(w * vy * 0x1p32));
    }
}

__global__ void regrid_finish_kernel(const unsigned long long* __restrict__ acc, int64_t n_nodes, double min_weight,
                                     double* __restrict__ out, double* __restrict__ weight)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_nodes) return;
    const long long qw = (long long)acc[3 * q];
    const double w = (double)qw * 0x1p-40;
    if (weight) weight[q] = w;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const bool keep = qw > 0 && w >= min_weight;
    const double inv = keep ? 0x1p8 / (double)qw : 0.0;    // 2^-32 px / (qw 2^-40)
    out[2 * q] = keep ? (double)(long long)acc[3 * q + 1] * inv : nan;
    out[2 * q + 1] = keep ? (double)(long long)acc[3 * q + 2] * inv : nan;
}

}  // namespace pivbos

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------

extern "C" {

pivbos_status pivbos_bos_displacements_range(const pivbos_medium* m, const pivbos_optics* o, const double* dots,
                                             int64_t n_dots, int64_t first_dot, int32_t rays_per_dot, uint64_t seed,
                                             uint32_t frame, int integrator, double step, double* centroid,
                                             double* displacement, int32_t* n_pairs, void* stream);

pivbos_status pivbos_bos_displacements(const pivbos_medium* m, const pivbos_optics* o, const double* dots,
                                       int64_t n_dots, int32_t rays_per_dot, uint64_t seed, uint32_t frame,
                                       int integrator, double step, double* centroid, double* displacement,
                                       int32_t* n_pairs, void* stream)
{
    return pivbos_bos_displacements_range(m, o, dots, n_dots, 0, rays_per_dot, seed, frame, integrator, step,
                                          centroid, displacement, n_pairs, stream);
}

pivbos_status pivbos_bos_displacements_range(const pivbos_medium* m, const pivbos_optics* o, const double* dots,
                                             int64_t n_dots, int64_t first_dot, int32_t rays_per_dot, uint64_t seed,
                                             uint32_t frame, int integrator, double step, double* centroid,
                                             double* displacement, int32_t* n_pairs, void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (!m) return failf(PIVBOS_ERR_INVALID_ARG, "medium handle is NULL");
    if (first_dot < 0 || first_dot + n_dots > 0xffffffffll)
        return failf(PIVBOS_ERR_INVALID_ARG, "first_dot %lld outside [0, 2^32 - n_dots]", (long long)first_dot);
    if (rays_per_dot > (1 << 22)) return failf(PIVBOS_ERR_UNSUPPORTED, "more than 2^22 rays per dot");
    TraceParams p;
    int dev;
    uint64_t total;
    pivbos_status st = prepare_trace(m, o, dots, n_dots, 1, rays_per_dot, seed, frame, integrator, step, &p, &dev,
                                     &total);
    if (st) return st;
    if (o->d.W > 65536 || o->d.H > 65536)
        return failf(PIVBOS_ERR_UNSUPPORTED, "sensor wider than 65536 pixels");
    if (n_dots == 0) return PIVBOS_OK;
    if (!centroid && !displacement && !n_pairs) return PIVBOS_OK;
    if (centroid && (st = device_pointer(centroid, dev, "centroid"))) return st;
    if (displacement && (st = device_pointer(displacement, dev, "displacement"))) return st;
    if (n_pairs && (st = device_pointer(n_pairs, dev, "n_pairs"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: per-slot sums | Morton keys | permutation | sorted dots (double-float)
    const uint32_t nd = (uint32_t)n_dots;
    uint32_t n_pow2 = 2;
    while (n_pow2 < nd) n_pow2 <<= 1;
    const size_t acc_bytes = (size_t)nd * kBosFields * sizeof(unsigned long long);
    const size_t off_keys = acc_bytes;
    const size_t off_perm = off_keys + (size_t)n_pow2 * 8;
    const size_t off_sdf = off_perm + (((size_t)nd * 4 + 255) & ~(size_t)255);
    const size_t bytes = off_sdf + (size_t)nd * 24;
    char* scratch = nullptr;
    if ((st = cuda_status(cudaMallocAsync((void**)&scratch, bytes, s), "displacement scratch"))) return st;
    unsigned long long* acc = (unsigned long long*)scratch;
    uint32_t* perm = (uint32_t*)(scratch + off_perm);
    float2* sdf = (float2*)(scratch + off_sdf);
    cudaError_t e = cudaMemsetAsync(acc, 0, acc_bytes, s);
    if (e == cudaSuccess) e = launch_morton_sort(dots, nd, (uint64_t*)(scratch + off_keys), n_pow2, perm, sdf, s);
    if (e == cudaSuccess && total > 0) {
        p.perm = perm;
        p.src_df = sdf;
        p.source_offset = (uint32_t)first_dot;
        const uint32_t rpc = rays_per_cta_setting(p);
        const uint64_t blocks = (total + rpc - 1) / rpc;
        timing_begin("bos_pairs", s);
        const unsigned g = (unsigned)blocks;
        const bool ext = optics_ext(p.o);
#define PV_BOS(I, C, E) bos_pairs_kernel<I, C, E><<<g, kBosThreads, 0, s>>>(p, acc, rpc, total)
        PV_DISPATCH(integrator, p.cell_cache != 0, ext, PV_BOS);
#undef PV_BOS
        timing_end("bos_pairs", s);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        bos_finish_kernel<<<(unsigned)((n_dots + 255) / 256), 256, 0, s>>>(acc, perm, n_dots, centroid, displacement,
                                                                          n_pairs);
        count_launches(1);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if ((st = cuda_status(e, "bos_displacements"))) return st;
    return cuda_status(ef, "displacement scratch release");
}

pivbos_status pivbos_bos_theory(const pivbos_medium* m, const pivbos_optics* o, const double* dots, int64_t n_dots,
                                double* displacement, void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (!m || !o) return failf(PIVBOS_ERR_INVALID_ARG, "medium or optics handle is NULL");
    if (n_dots < 0 || n_dots > (1ll << 31)) return failf(PIVBOS_ERR_INVALID_ARG, "n_dots %lld", (long long)n_dots);
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status(cudaGetLastError(), "cudaGetDevice");
    if (m->device != dev || o->device != dev)
        return failf(PIVBOS_ERR_INVALID_ARG, "handles belong to another device");
    if (n_dots == 0) return PIVBOS_OK;
    pivbos_status st;
    if ((st = device_pointer(dots, dev, "dots"))) return st;
    if ((st = device_pointer(displacement, dev, "displacement"))) return st;
    Eq9Geom G;
    G.field = m->field;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = m->n[a];
        G.origin[a] = m->origin[a];
        G.h[a] = m->spacing[a];
    }
    G.aim_z = o->aim_z;
    G.scale = o->magnification / (o->n_object * o->pixel_pitch);
    G.z_mid = m->origin[2] + 0.5 * (double)(m->n[2] - 1) * m->spacing[2];
    cudaStream_t s = (cudaStream_t)stream;
    timing_begin("bos_theory", s);
    bos_theory_kernel<<<(unsigned)((n_dots + 127) / 128), 128, 0, s>>>(G, dots, n_dots, displacement);
    timing_end("bos_theory", s);
    count_launches(1);
    return cuda_status(cudaGetLastError(), "bos_theory");
}

pivbos_status pivbos_regrid_bilinear(const double* xy, const double* values, int64_t n, int grid_w, int grid_h,
                                     double x0, double y0, double cell, double min_weight, double* out,
                                     double* weight, void* stream)
{
    using namespace pivbos;
    set_last_error("");
    if (n < 0 || n > (1ll << 23)) return failf(PIVBOS_ERR_INVALID_ARG, "n %lld outside [0, 2^23]", (long long)n);
    if (grid_w < 2 || grid_h < 2 || (int64_t)grid_w * grid_h > (1ll << 28))
        return failf(PIVBOS_ERR_INVALID_ARG, "grid %d x %d", grid_w, grid_h);
    if (!(isfinite(x0) && isfinite(y0) && isfinite(cell) && cell > 0.0) || !(min_weight >= 0.0))
        return failf(PIVBOS_ERR_INVALID_ARG, "grid origin, cell or min_weight");
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status(cudaGetLastError(), "cudaGetDevice");
    pivbos_status st;
    if ((st = device_pointer(out, dev, "out"))) return st;
    if (weight && (st = device_pointer(weight, dev, "weight"))) return st;
    if (n > 0) {
        if ((st = device_pointer(xy, dev, "xy"))) return st;
        if ((st = device_pointer(values, dev, "values"))) return st;
    }
    int* sw = nullptr;
    if ((st = device_status_word(dev, &sw))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nodes = (int64_t)grid_w * grid_h;
    const size_t bytes = (size_t)nodes * 3 * sizeof(unsigned long long);
    unsigned long long* acc = nullptr;
    if ((st = cuda_status(cudaMallocAsync((void**)&acc, bytes, s), "regrid accumulators"))) return st;
    cudaError_t e = cudaMemsetAsync(acc, 0, bytes, s);
    if (e == cudaSuccess && n > 0) {
        timing_begin("regrid", s);
        regrid_splat_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xy, values, n, grid_w, grid_h, x0, y0,
                                                                       1.0 / cell, acc, sw);
        timing_end("regrid", s);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        regrid_finish_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(acc, nodes, min_weight, out, weight);
        count_launches(1);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(acc, s);
    if ((st = cuda_status(e, "regrid_bilinear"))) return st;
    return cuda_status(ef, "regrid accumulators release");
}

}  // extern "C"
