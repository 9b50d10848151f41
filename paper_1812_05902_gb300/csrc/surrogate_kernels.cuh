// Device side of the surrogate ray map (no counterpart in the paper: a
// learned part built on the tracer of Sec. 3.2): the projection table and
// its lookups, training data and confidence-map kernels, and the render
// kernels (prep -> tcgen05 network -> finish).  Host code in surrogate.cu.
#pragma once

#include <cuda_bf16.h>

#include "mlp_tc.cuh"
#include "trace.cuh"

namespace pivbos {

// Geometry and normalisation of one trained surrogate (device copy).
struct SurrParams {
    dfc z_lo;                       // box front (entry plane for sources in front of the box)
    dfc z_ref;                      // reference plane of the exit-line residual
    float cx, cy, cz, hx, hy, hz;   // box centre and half extents (feature scaling)
    float u_scale;                  // slope scaling
    float inv_h[3], inv_u_scale;    // 1 / hx, 1 / hy, 1 / hz, 1 / u_scale
    float inv_b_scale[4];           // 1 / b_scale
    float t_scale[4];               // network output scales: dx, dy (m) at z_ref, dux, duy
    float b_scale[4];               // scales of the projection (Born) residual as network input
    int nbx, nby, nbz, nbu;         // confidence bins
    const uint32_t* bin_ok;         // bit b set: bin b is served (not traced by the plain path)
    const uint32_t* bin_net;        // bit b set: bin b is served with the network's correction (use_net 2)
    int use_net;                    // 0: the projection residual alone; 1: with the network's correction in
                                    // every served bin; 2: in the bins of bin_net only
    // projection table: suffix integrals of grad n along lines through the
    // pupil centre (0, 0, aim_z), columns indexed by where they cross z_hi
    const float4* table;            // G plane [level][row][col] {Gx, Gy, Gz, 0}, then the H plane
    const float4* table_h;          //   {Hx, Hy, Hz, 0} (= table + nodes)
    int tnx, tny, tnz, born_k;      // columns, levels; segments per ray (0: no projection)
    float t_x0, t_y0, t_inv_dx, t_inv_dy, t_inv_dz;
    float zlo_f, zhi_f, aim_z, persp;   // persp = aim_z - z_hi
};

constexpr int kSurrBins = 16 * 16 * 16 * 4 * 4;

struct Entry {
    bool enters;
    float f[5];    // entry x, y, z, slope x, slope y (scaled to about [-1, 1])
    int bin;
    float xs, ys;  // straight line at the reference plane
    float ux, uy;  // slopes dx/dz, dy/dz of the straight ray
    float xe, ye, ze;   // entry point (m)
};

__device__ __forceinline__ int bin_of(float f, int nb)
{
    const int b = (int)floorf((f + 1.0f) * 0.5f * (float)nb);
    return min(max(b, 0), nb - 1);
}

// The surrogate path's ray in FP32: the lens point from the same Philox
// words as the plain path (Sec. 3.1), rounded to FP32 (the surrogate's model
// error, ~1e-3 px, is far above what FP32 rays change: ~1e-5 px).
__device__ __forceinline__ void ray_start_f(const TraceParams& P, float sx, float sy, float sz, uint32_t sid,
                                            uint32_t rid, float& dx, float& dy, float& dz)
{
    uint64_t w0, w1;
    philox_lens_words(rid, sid, P.frame, 0ull, P.seed, 0ull, w0, w1);
    const df u1 = u01_df(w0), u2 = u01_df(w1);
    const float r = (P.o.aim_r.hi + P.o.aim_r.lo) * sqrtf(u1.hi + u1.lo);
    float sn, cs;
    sincospif(2.0f * (u2.hi + u2.lo), &sn, &cs);
    dx = r * cs - sx;
    dy = r * sn - sy;
    dz = (P.o.aim_z.hi + P.o.aim_z.lo) - sz;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
}

// Whether the straight ray meets the box (slab test, FP32).
__device__ __forceinline__ bool box_entry_f(const DevMedium& m, float Rx, float Ry, float Rz, float dx, float dy,
                                            float dz)
{
    const float R[3] = {Rx, Ry, Rz}, d[3] = {dx, dy, dz};
    float t_near = 0.0f, t_far = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = m.lo[a].hi + m.lo[a].lo, hi = m.hi[a].hi + m.hi[a].lo;
        if (d[a] == 0.0f) {
            if (R[a] < lo || R[a] > hi) return false;
        } else {
            const float inv = 1.0f / d[a];
            const float t1 = (lo - R[a]) * inv, t2 = (hi - R[a]) * inv;
            t_near = fmaxf(t_near, fminf(t1, t2));
            t_far = fminf(t_far, fmaxf(t1, t2));
        }
    }
    return t_near <= t_far;
}

// Entry state of the FP32 ray of (source s, ray k): the straight line's
// point on the plane z = max(z_lo, s_z) and its slopes (the network's
// features), the confidence bin, and the straight line at the reference
// plane.
__device__ __forceinline__ void surr_entry_f(const TraceParams& P, const SurrParams& S, float sx, float sy, float sz,
                                             uint32_t sid, uint32_t k, Entry& e)
{
    float dx, dy, dz;
    ray_start_f(P, sx, sy, sz, sid, k, dx, dy, dz);
    e.enters = box_entry_f(P.m, sx, sy, sz, dx, dy, dz);
    const float idz = 1.0f / dz;
    const float ux = dx * idz, uy = dy * idz;
    const float zlo = S.z_lo.hi + S.z_lo.lo, zr = S.z_ref.hi + S.z_ref.lo;
    const float ze = sz < zlo ? zlo : sz;
    e.xe = fmaf(ux, ze - sz, sx);
    e.ye = fmaf(uy, ze - sz, sy);
    e.ze = ze;
    e.ux = ux;
    e.uy = uy;
    e.xs = fmaf(ux, zr - sz, sx);
    e.ys = fmaf(uy, zr - sz, sy);
    e.f[0] = (e.xe - S.cx) * S.inv_h[0];
    e.f[1] = (e.ye - S.cy) * S.inv_h[1];
    e.f[2] = (ze - S.cz) * S.inv_h[2];
    e.f[3] = ux * S.inv_u_scale;
    e.f[4] = uy * S.inv_u_scale;
    const int bu = bin_of(e.f[3], S.nbu) * S.nbu + bin_of(e.f[4], S.nbu);
    e.bin = ((bin_of(e.f[0], S.nbx) * S.nby + bin_of(e.f[1], S.nby)) * S.nbz + bin_of(e.f[2], S.nbz)) *
                (S.nbu * S.nbu) + bu;
}

// Source (FP64 as given -> double-float) and FP32 entry state of a ray by id.
__device__ __forceinline__ void surr_ray_by_id(const TraceParams& P, const SurrParams& S, uint64_t id, uint32_t& sid,
                                               uint32_t& k, df& sx, df& sy, df& sz, Entry& e)
{
    const uint32_t rps = P.rays_per_source;
    sid = (uint32_t)(id / rps);
    k = (uint32_t)(id - (uint64_t)sid * rps);
    const double* sp = P.sources + 3 * (size_t)sid;
    sx = df_from_double(sp[0]);
    sy = df_from_double(sp[1]);
    sz = df_from_double(sp[2]);
    surr_entry_f(P, S, sx.hi + sx.lo, sy.hi + sy.lo, sz.hi + sz.lo, sid + P.source_offset, k, e);
}

// Table value at column coordinates (xi, eta) and depth z: bilinear across
// columns, linear across levels; zero for columns outside the table (lines
// that miss the box).  H only when WANT_H.
template <bool WANT_H>
__device__ __forceinline__ void table_lookup(const SurrParams& S, float xi, float eta, float z, float3& G, float3& H)
{
    const float fx = (xi - S.t_x0) * S.t_inv_dx, fy = (eta - S.t_y0) * S.t_inv_dy;
    G = make_float3(0.f, 0.f, 0.f);
    H = make_float3(0.f, 0.f, 0.f);
    if (!(fx >= 0.0f && fy >= 0.0f && fx <= (float)(S.tnx - 1) && fy <= (float)(S.tny - 1))) return;
    const float fz = fminf(fmaxf((z - S.zlo_f) * S.t_inv_dz, 0.0f), (float)(S.tnz - 1));
    const int i = min((int)fx, S.tnx - 2), j = min((int)fy, S.tny - 2), l = min((int)fz, S.tnz - 2);
    const float ax = fx - (float)i, ay = fy - (float)j, az = fz - (float)l;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dl = c >> 2;
        const float w = (di ? ax : 1.0f - ax) * (dj ? ay : 1.0f - ay) * (dl ? az : 1.0f - az);
        const size_t node = ((size_t)(l + dl) * S.tny + (j + dj)) * S.tnx + (i + di);
        const float4 g = __ldg(S.table + node);
        G.x = fmaf(w, g.x, G.x); G.y = fmaf(w, g.y, G.y); G.z = fmaf(w, g.z, G.z);
        if constexpr (WANT_H) {
            const float4 h = __ldg(S.table_h + node);
            H.x = fmaf(w, h.x, H.x); H.y = fmaf(w, h.y, H.y); H.z = fmaf(w, h.z, H.z);
        }
    }
}

// Projection (Born-type) exit-line residual of a ray from its entry point
// with straight slopes (ux, uy): dT/ds = grad n (the ray equation with
// dt = ds / n) integrated along the line cut into born_k segments, each
// segment's integrals taken from the table column through the segment's
// midpoint.  The midpoint is moved by the displacement the earlier segments
// have already produced, so the integrals follow the deflected path
// (first-order accurate in each segment, self-consistent along the ray).
// With 8 or more segments a segment's first moment H is taken as its
// midpoint offset times G (the table's H plane is read only for fewer,
// longer segments).  r = {dx, dy at z_ref, dux, duy}.
__device__ __forceinline__ void born_residual(const SurrParams& S, const Entry& e, float* r)
{
    r[0] = r[1] = r[2] = r[3] = 0.0f;
    if (S.born_k <= 0 || !e.enters) return;
    const float ux = e.ux, uy = e.uy;
    const float q = 1.0f + ux * ux + uy * uy;   // slope change (T_perp - u T_z) / T_z with T = n d, ds = dz sqrt(1+u^2)
    const float dzs = (S.zhi_f - e.ze) / (float)S.born_k;
    // accumulated slope-change integrals of the segments done so far:
    // gx, gy = sum of (G_perp - u G_z); hx, hy = the same with weight (z - z_hi)
    float gx = 0.f, gy = 0.f, hx = 0.f, hy = 0.f;
#pragma unroll 1
    for (int k = 0; k < S.born_k; ++k) {
        const float za = e.ze + (float)k * dzs, zb = za + dzs, zm = za + 0.5f * dzs;
        // displacement at zm from the earlier segments' kinks
        const float dxm = q * ((zm - S.zhi_f) * gx - hx), dym = q * ((zm - S.zhi_f) * gy - hy);
        const float c = S.persp / (S.aim_z - zm);
        const float xi = (e.xe + ux * (zm - e.ze) + dxm) * c, eta = (e.ye + uy * (zm - e.ze) + dym) * c;
        // the last segment ends on the box's far face, the table's top level,
        // where the integrals start: zero there, not read
        const bool last = k == S.born_k - 1;
        float3 Ga, Ha, Gb = make_float3(0.f, 0.f, 0.f), Hb = Gb;
        float Hx, Hy, Hz;
        if (S.born_k >= 8) {
            table_lookup<false>(S, xi, eta, za, Ga, Ha);
            if (!last) table_lookup<false>(S, xi, eta, zb, Gb, Hb);
            const float zo = zm - S.zhi_f;
            Hx = zo * (Ga.x - Gb.x); Hy = zo * (Ga.y - Gb.y); Hz = zo * (Ga.z - Gb.z);
        } else {
            table_lookup<true>(S, xi, eta, za, Ga, Ha);
            if (!last) table_lookup<true>(S, xi, eta, zb, Gb, Hb);
            Hx = Ha.x - Hb.x; Hy = Ha.y - Hb.y; Hz = Ha.z - Hb.z;
        }
        const float Gx = Ga.x - Gb.x, Gy = Ga.y - Gb.y, Gz = Ga.z - Gb.z;
        gx += Gx - ux * Gz;
        gy += Gy - uy * Gz;
        hx += Hx - ux * Hz;
        hy += Hy - uy * Hz;
    }
    const float zr = S.z_ref.hi + S.z_ref.lo - S.zhi_f;
    r[0] = q * (zr * gx - hx);
    r[1] = q * (zr * gy - hy);
    r[2] = q * gx;
    r[3] = q * gy;
}

// Network input: each entry feature as a BF16 value and its BF16-rounded
// remainder times 256 (16 significant bits in all), then the scaled
// projection residual, zero padded.
__device__ __forceinline__ void encode_features(const SurrParams& S, const float* f, const float* born,
                                                __nv_bfloat16* x)
{
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const __nv_bfloat16 hi = __float2bfloat16(f[c]);
        x[c] = hi;
        x[5 + c] = __float2bfloat16((f[c] - __bfloat162float(hi)) * 256.0f);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) x[10 + c] = __float2bfloat16(born[c] * S.inv_b_scale[c]);
    x[14] = x[15] = __float2bfloat16(0.0f);
}

// Exit line from the residual r (m, m, rad, rad): a point on the reference
// plane and the unit direction, in double-float (the pilot's finite
// differences of the sensor position).
__device__ __forceinline__ void surr_exit(const SurrParams& S, const Entry& e, const float* r, df& Rx, df& Ry, df& Rz,
                                          df& dx, df& dy, df& dz)
{
    Rx = df_add_f(dfv(e.xs), r[0]);
    Ry = df_add_f(dfv(e.ys), r[1]);
    Rz = dfk(S.z_ref);
    const df ux = df_add_f(dfv(e.ux), r[2]);
    const df uy = df_add_f(dfv(e.uy), r[3]);
    const df inn = df_rsqrt(df_add_f(df_add(df_sqr(ux), df_sqr(uy)), 1.0f));
    dx = df_mul(ux, inn);
    dy = df_mul(uy, inn);
    dz = inn;
}

// Whether served rays of bin b take the network's correction.
__device__ __forceinline__ bool net_bin(const SurrParams& S, int b)
{
    if (S.use_net == 2) return (__ldg(S.bin_net + (b >> 5)) >> (b & 31)) & 1u;
    return S.use_net == 1;
}

// Full residual: projection plus (with net) the network's correction (y scaled).
__device__ __forceinline__ void surr_residual(const SurrParams& S, const float* born, const float* y, bool net,
                                              float* r)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) r[c] = born[c] + (net ? y[c] * S.t_scale[c] : 0.0f);
}

// Sensor position of a surrogate ray: its straight line (xs, ys at z_ref,
// slopes ux, uy) plus the residual r gives the exit line, which passes the
// lens and reaches the sensor in FP32 (the surrogate's own error, ~1e-3 px,
// is far above their rounding; the plain path keeps double-float optics for
// its 1e-5 px parity).  status: PIVBOS_RAY_REACHED on entry.
template <bool EXT = true>
__device__ __forceinline__ void surr_sensor(const DevOptics& o, const SurrParams& S, float xs, float ys, float ux,
                                            float uy, const float* r, int& status, df& px, df& py)
{
    float x = xs + r[0], y = ys + r[1], z = S.z_ref.hi + S.z_ref.lo;
    const float vx = ux + r[2], vy = uy + r[3];
    const float inn = rsqrtf(fmaf(vx, vx, fmaf(vy, vy, 1.0f)));
    float dx = vx * inn, dy = vy * inn, dz = inn;
    float fx, fy;
    optics_to_sensor<F32Ops, EXT>(o, x, y, z, dx, dy, dz, status, fx, fy);
    px = dfv(fx);
    py = dfv(fy);
}

// Seeded sample of ray ids of a frame (Philox counter (q, stream, frame, 2)).
__device__ __forceinline__ uint64_t sample_ray(const TraceParams& P, uint64_t q, uint32_t stream, uint64_t seed,
                                               uint64_t total)
{
    uint64_t w0, w1;
    philox_lens_words(q, stream, P.frame, 2ull, seed, 0ull, w0, w1);
    return w0 % total;
}

// Projection table: one thread per column; the column's line is followed
// from z_hi down to z_lo, grad n sampled (trilinear, as the tracer samples
// it; zero outside the box) at the midpoints of `sub` sub-steps per level.
__global__ void surr_table_kernel(const DevMedium m, SurrParams S, int sub, float4* __restrict__ table)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= S.tnx * S.tny) return;
    const int i = col % S.tnx, j = col / S.tnx;
    const float xi = S.t_x0 + (float)i / S.t_inv_dx, eta = S.t_y0 + (float)j / S.t_inv_dy;
    const double lo0 = m.lo[0].hi + (double)m.lo[0].lo, hi0 = m.hi[0].hi + (double)m.hi[0].lo;
    const double lo1 = m.lo[1].hi + (double)m.lo[1].lo, hi1 = m.hi[1].hi + (double)m.hi[1].lo;
    const double ox = m.origin[0].hi + (double)m.origin[0].lo, oy = m.origin[1].hi + (double)m.origin[1].lo;
    const double oz = m.origin[2].hi + (double)m.origin[2].lo;
    const double dzl = 1.0 / S.t_inv_dz, h = dzl / sub;
    double G[3] = {0, 0, 0}, H[3] = {0, 0, 0};
    for (int l = S.tnz - 1; l >= 0; --l) {
        if (l < S.tnz - 1) {
            const double zt = S.zlo_f + (double)(l + 1) * dzl;
            for (int q = 0; q < sub; ++q) {
                const double z = zt - (q + 0.5) * h;
                const double c = (S.aim_z - z) / S.persp;
                const double x = xi * c, y = eta * c;
                if (x < lo0 || x > hi0 || y < lo1 || y > hi1) continue;
                const float4 v = sample_field(m, (float)((x - ox) * m.inv_h[0]), (float)((y - oy) * m.inv_h[1]),
                                              (float)((z - oz) * m.inv_h[2]));
                const double wz = (z - S.zhi_f) * h;
                G[0] += v.y * h; G[1] += v.z * h; G[2] += v.w * h;
                H[0] += v.y * wz; H[1] += v.z * wz; H[2] += v.w * wz;
            }
        }
        const size_t node = ((size_t)l * S.tny + j) * S.tnx + i;
        table[node] = make_float4((float)G[0], (float)G[1], (float)G[2], 0.f);
        table[(size_t)S.tnx * S.tny * S.tnz + node] = make_float4((float)H[0], (float)H[1], (float)H[2], 0.f);
    }
}

// Truth (plain path) and projection residuals of one ray.
template <int INTEG>
__device__ __forceinline__ void truth_and_born(const TraceParams& P, const SurrParams& S, uint64_t id, Entry& e,
                                               pivbos_ray_state& st, float* t, float* born)
{
    uint32_t sid, k;
    df sx, sy, sz;
    surr_ray_by_id(P, S, id, sid, k, sx, sy, sz, e);
    born_residual(S, e, born);
    RayOut r;
    trace_ray<INTEG, false>(P, sx, sy, sz, sid + P.source_offset, k, r, &st);   // the plain path's ray
    t[0] = t[1] = t[2] = t[3] = 0.0f;
    if (st.status != PIVBOS_RAY_MAXSTEP) {
        // the exit line (straight beyond the box) against the surrogate's
        // straight ray, both taken at the reference plane
        const double zr = df_to_double(dfk(S.z_ref));
        const double Dx = st.vol_dir[0] / st.vol_dir[2], Dy = st.vol_dir[1] / st.vol_dir[2];
        const double xt = st.vol_pos[0] + (zr - st.vol_pos[2]) * Dx;
        const double yt = st.vol_pos[1] + (zr - st.vol_pos[2]) * Dy;
        t[0] = (float)(xt - (double)e.xs);
        t[1] = (float)(yt - (double)e.ys);
        t[2] = (float)(Dx - (double)e.ux);
        t[3] = (float)(Dy - (double)e.uy);
    }
}

// Pilot statistics on a few rays: mean squares of the truth residual, of
// the projection residual and of their difference ([0..11]), the sensor
// shift per unit of each residual component by finite differences about
// the straight ray ([12..15], [16] = rays counted), and for each candidate
// segment count kc = 1, 2, 4, ..., the squared sensor error of the
// projection alone against the plain path ([17 + c], [17 + kPilotK] =
// rays compared).
constexpr int kPilotK = 6;   // candidates 1, 2, 4, 8, 16, 32

template <int INTEG>
__global__ void surr_pilot_kernel(const TraceParams P, const SurrParams S, uint64_t total, int64_t n, uint64_t seed,
                                  double dpos, double dslope, double* __restrict__ acc)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int NV = 18 + kPilotK;
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    if (q < n) {
        Entry e;
        pivbos_ray_state st;
        float t[4], born[4];
        truth_and_born<INTEG>(P, S, sample_ray(P, (uint64_t)q, 3, seed, total), e, st, t, born);
        for (int c = 0; c < 4; ++c) {
            v[c] = (double)t[c] * t[c];
            v[4 + c] = (double)born[c] * born[c];
            v[8 + c] = (double)(t[c] - born[c]) * (t[c] - born[c]);
        }
        double px[5], py[5];
        bool ok = true;
#pragma unroll 1
        for (int c = 0; c < 5; ++c) {
            float r[4] = {0.f, 0.f, 0.f, 0.f};
            if (c > 0) r[c - 1] = (float)(c <= 2 ? dpos : dslope);
            df Rx, Ry, Rz, ex, ey, ez;
            surr_exit(S, e, r, Rx, Ry, Rz, ex, ey, ez);
            int status = PIVBOS_RAY_REACHED;
            df a, b;
            optics_to_sensor(P.o, Rx, Ry, Rz, ex, ey, ez, status, a, b);
            ok = ok && status == PIVBOS_RAY_REACHED;
            px[c] = df_to_double(a);
            py[c] = df_to_double(b);
        }
        if (ok) {
            for (int c = 1; c < 5; ++c) {
                const double d = c <= 2 ? dpos : dslope;
                const double ax = px[c] - px[0], ay = py[c] - py[0];
                v[11 + c] = (ax * ax + ay * ay) / (d * d);
            }
            v[16] = 1.0;
        }
        if (S.born_k != 0 && e.enters && st.status == PIVBOS_RAY_REACHED) {
            bool all = true;
            double err[kPilotK];
#pragma unroll 1
            for (int c = 0; c < kPilotK; ++c) {
                SurrParams Sk = S;
                Sk.born_k = 1 << c;
                float r[4];
                born_residual(Sk, e, r);
                int status = PIVBOS_RAY_REACHED;
                df a, b;
                surr_sensor(P.o, S, e.xs, e.ys, e.ux, e.uy, r, status, a, b);
                all = all && status == PIVBOS_RAY_REACHED;
                const double dx = df_to_double(a) - st.sensor_xy[0], dy = df_to_double(b) - st.sensor_xy[1];
                err[c] = dx * dx + dy * dy;
            }
            if (all) {
                for (int c = 0; c < kPilotK; ++c) v[17 + c] = err[c];
                v[17 + kPilotK] = 1.0;
            }
        }
    }
    for (int c = 0; c < NV; ++c) {
        for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
        if ((threadIdx.x & 31) == 0 && v[c] != 0.0) atomicAdd(&acc[c], v[c]);
    }
}

// S1: samples of (encoded entry features and projection residual, scaled
// correction truth - projection) traced by the plain path.  For held-out
// samples also the plain sensor position, status and step count.
template <int INTEG>
__global__ void surr_data_kernel(const TraceParams P, const SurrParams S, uint64_t total, int64_t n, uint32_t stream,
                                 uint64_t seed, __nv_bfloat16* __restrict__ X, float* __restrict__ T,
                                 uint64_t* __restrict__ ids, double* __restrict__ ref_px, int* __restrict__ ref_st)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint64_t id = sample_ray(P, (uint64_t)q, stream, seed, total);
    Entry e;
    pivbos_ray_state st;
    float t[4], born[4];
    truth_and_born<INTEG>(P, S, id, e, st, t, born);
    encode_features(S, e.f, born, X + (size_t)q * kMlpIn);
    if (T)
        *reinterpret_cast<float4*>(T + (size_t)q * 4) =
            make_float4((t[0] - born[0]) / S.t_scale[0], (t[1] - born[1]) / S.t_scale[1],
                        (t[2] - born[2]) / S.t_scale[2], (t[3] - born[3]) / S.t_scale[3]);
    if (ids) ids[q] = id;
    if (ref_px) {
        ref_px[2 * q] = st.sensor_xy[0];
        ref_px[2 * q + 1] = st.sensor_xy[1];
        ref_st[q] = st.status | (st.steps << 3);
    }
}

// Per-bin sums over held-out rays that reach the sensor in the plain path,
// for three predictors: the network (projection + correction), the
// projection alone, and the straight ray.
struct BinAcc {
    double* err2[3];     // squared sensor error (px^2) per predictor
    double* steps;       // plain-path integration steps (the work a served ray saves)
    unsigned int* cnt;
    double* tot;         // [0] rays reaching the sensor, [1] those entering the box,
                         // [2..4] of these, rays each predictor sends elsewhere
};

// Confidence map: the plain tracer judges each predictor at the sensor.
// A ray whose status differs from the plain path's (one grazing a stop)
// has no displacement: it is counted, not summed.
__global__ void surr_eval_kernel(const TraceParams P, const SurrParams S, const uint64_t* __restrict__ ids,
                                 const float* __restrict__ Y, const double* __restrict__ ref_px,
                                 const int* __restrict__ ref_st, int64_t n, BinAcc acc)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    if ((ref_st[q] & 7) != PIVBOS_RAY_REACHED) return;
    atomicAdd(&acc.tot[0], 1.0);
    uint32_t sid, k;
    df sx, sy, sz;
    Entry e;
    surr_ray_by_id(P, S, ids[q], sid, k, sx, sy, sz, e);
    if (!e.enters) return;
    atomicAdd(&acc.tot[1], 1.0);
    float born[4], y[4];
    born_residual(S, e, born);
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = Y[q * 4 + c];
#pragma unroll 1
    for (int v = 0; v < 3; ++v) {
        float r[4] = {0.f, 0.f, 0.f, 0.f};
        if (v == 0) {
            for (int c = 0; c < 4; ++c) r[c] = born[c] + y[c] * S.t_scale[c];
        } else if (v == 1) {
            for (int c = 0; c < 4; ++c) r[c] = born[c];
        }
        int status = PIVBOS_RAY_REACHED;
        df px, py;
        surr_sensor(P.o, S, e.xs, e.ys, e.ux, e.uy, r, status, px, py);
        if (status == PIVBOS_RAY_REACHED) {
            const double a = df_to_double(px) - ref_px[2 * q], b = df_to_double(py) - ref_px[2 * q + 1];
            atomicAdd(&acc.err2[v][e.bin], a * a + b * b);
        } else {
            atomicAdd(&acc.tot[2 + v], 1.0);
        }
    }
    atomicAdd(&acc.steps[e.bin], (double)(ref_st[q] >> 3));
    atomicAdd(&acc.cnt[e.bin], 1u);
}

// ---------------------------------------------------------------------------
// Surrogate render in three kernels over chunks of the frame's rays:
// prep (features, projection, serve / fall back) -> network (tcgen05) ->
// finish (exit line, optics, tile deposit).  Each runs at its own
// occupancy; the served rays pass between them in ray order.
// ---------------------------------------------------------------------------
struct ServedList {
    uint32_t* ids;              // flat ray index; top bit: never enters the box (straight)
    __nv_bfloat16* X;           // [capacity][16] network input (by network slot)
    float4* B;                  // [capacity] projection residual (by network slot with use_net 1 and 2,
                                // by served slot with use_net 0)
    float4* R;                  // [capacity] full residual (projection + correction), by served slot
    float4* L;                  // [capacity] straight line: x, y at z_ref and slopes x, y
    unsigned long long* count;  // rays appended
    uint32_t capacity;
    // use_net 2: the rays that take the network's correction, a sub-list of
    // the served list (network slot -> served slot); nullptr: every served
    // ray, network slot = served slot
    uint32_t* net_idx;
    unsigned long long* net_count;
};

constexpr uint32_t kStraightBit = 0x80000000u;

// Append the calling CTA's lanes to one of two lists (flag a: list A, flag
// b: list B; at most one of them set per lane), with one atomic per CTA and
// list; returns this thread's slot in its list (meaningful where a flag is
// set).  All threads call it; blockDim.x <= 256.
__device__ __forceinline__ unsigned long long block_append2(bool fa, bool fb, unsigned long long* count_a,
                                                            unsigned long long* count_b, int (*warp_off)[8],
                                                            unsigned long long* base)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    const unsigned ma = __ballot_sync(0xffffffffu, fa), mb = __ballot_sync(0xffffffffu, fb);
    __syncthreads();   // every thread has read the previous call's offsets
    if (lane == 0) {
        warp_off[0][warp] = __popc(ma);
        warp_off[1][warp] = __popc(mb);
    }
    __syncthreads();
    if (tid < 2) {
        int tot = 0;
        for (int w = 0; w < nw; ++w) {
            const int c = warp_off[tid][w];
            warp_off[tid][w] = tot;
            tot += c;
        }
        base[tid] = tot ? atomicAdd(tid ? count_b : count_a, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    const int l = fb ? 1 : 0;
    const unsigned m = fb ? mb : ma;
    return base[l] + (unsigned long long)(warp_off[l][warp] + __popc(m & ((1u << lane) - 1u)));
}

// Prep: rays [c0, c1) of the Morton-ordered (slot, ray) space, 256 per CTA
// round; served rays (and rays that never enter the box) go to the served
// list with their network input and projection residual, the others to the
// fallback list.
__global__ void __launch_bounds__(256)
surr_prep_kernel(const TraceParams P, const SurrParams S, uint64_t c0, uint64_t c1, ServedList sv,
                 uint32_t* __restrict__ fb_ids, unsigned long long* __restrict__ fb_count, uint32_t fb_capacity)
{
    __shared__ int warp_off[2][8];
    __shared__ unsigned long long base[2];
    __shared__ int warp_off_n[2][8];
    __shared__ unsigned long long base_n[2];
    __shared__ uint32_t order[kMaxOrderRays];
    const uint32_t rps = P.rays_per_source;
    // items of kMaxOrderRays rays; with many projection segments per ray an
    // item's rays are taken in the order of where they cross the box
    // mid-plane, so a warp's table gathers share columns
    const uint64_t items = (c1 - c0 + kMaxOrderRays - 1) / kMaxOrderRays;
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint64_t first = c0 + it * kMaxOrderRays;
        const uint32_t n_here = (uint32_t)(min(first + kMaxOrderRays, c1) - first);
        const bool reorder = P.reorder && S.born_k >= 8;
        if (reorder) order_chunk(P, order, first, n_here);
        for (uint32_t r0 = 0; r0 < n_here; r0 += 256) {
            const uint32_t pos = r0 + threadIdx.x;
            const bool active = pos < n_here;
            const uint64_t idx = first + (reorder && active ? (order[pos] & 0x7ffu) : pos);
            int mode = 3;
            bool net = false;
            Entry e;
            e.enters = false;
            e.f[0] = e.f[1] = e.f[2] = e.f[3] = e.f[4] = 0.0f;
            float born[4] = {0.f, 0.f, 0.f, 0.f};
            if (active) {
                const uint32_t flat = (uint32_t)idx;
                const uint32_t slot = flat / rps, k = flat - slot * rps;
                const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
                const float2* sp = P.src_df + 3 * (size_t)slot;
                const float2 a = __ldg(sp), b = __ldg(sp + 1), c = __ldg(sp + 2);
                surr_entry_f(P, S, a.x + a.y, b.x + b.y, c.x + c.y, sid, k, e);
                if (!e.enters) mode = 2;
                else mode = ((__ldg(S.bin_ok + (e.bin >> 5)) >> (e.bin & 31)) & 1u) ? 0 : 1;
                if (mode == 0) {
                    born_residual(S, e, born);
                    net = net_bin(S, e.bin);
                }
                // use_net 1 runs the network over the whole served list
                // (a straight ray's result is not read)
                if (mode == 2 && S.use_net == 1) net = true;
            }
            // served and straight rays to the served list, the rest to the
            // fallback list
            const unsigned long long ps = block_append2(mode == 0 || mode == 2, mode == 1, sv.count, fb_count,
                                                        warp_off, base);
            // use_net 2: the served rays that take the network's correction
            // to the network's sub-list as well
            unsigned long long pn = ps;
            if (S.use_net == 2) pn = block_append2(net, false, sv.net_count, sv.net_count, warp_off_n, base_n);
            if (mode == 0 || mode == 2) {
                if (ps < sv.capacity && (!net || pn < sv.capacity)) {
                    // streaming stores: the lists pass through HBM once,
                    // leaving L2 to the projection table
                    __stcs(sv.ids + ps, (uint32_t)idx | (mode == 2 ? kStraightBit : 0u));
                    const float4 b4 = make_float4(born[0], born[1], born[2], born[3]);
                    if (net) {
                        __align__(16) __nv_bfloat16 x[kMlpIn];
                        encode_features(S, e.f, born, x);
                        uint4* xr = reinterpret_cast<uint4*>(sv.X + pn * kMlpIn);
                        __stcs(xr, *reinterpret_cast<const uint4*>(&x[0]));
                        __stcs(xr + 1, *reinterpret_cast<const uint4*>(&x[8]));
                        __stcs(sv.B + pn, b4);
                        if (S.use_net == 2) __stcs(sv.net_idx + pn, (uint32_t)ps);
                    }
                    if (S.use_net == 0) __stcs(sv.B + ps, b4);
                    else if (!net) __stcs(sv.R + ps, b4);   // the projection alone (or a straight ray)
                    __stcs(sv.L + ps, make_float4(e.xs, e.ys, e.ux, e.uy));
                } else {
                    atomicCAS(P.status_word, 0, (int)PIVBOS_ERR_OVERFLOW);   // cannot happen: capacity = chunk
                }
            }
            if (mode == 1) {
                if (ps < fb_capacity) fb_ids[ps] = (uint32_t)idx;
                else atomicCAS(P.status_word, 0, (int)PIVBOS_ERR_OVERFLOW);   // cannot happen: capacity = rays
            }
        }
        __syncthreads();   // order[] is rewritten by the next item
    }
}

// Network over the served list on tcgen05: two warpgroups per CTA, each
// running its own 128-row tiles (TMEM columns [256g, 256g + 256), its own
// mbarrier), so one tile's MMAs overlap the other's epilogue; the next
// tile's inputs are loaded during the current one.  R = B + y * scale.
constexpr int kNetGroups = 2;
struct NetSmem {
    mlptc::Net net;
    uint64_t bar[kNetGroups];
    uint32_t tmem_base;
};

__global__ void __launch_bounds__(128 * kNetGroups, 1)
surr_net_kernel(const SurrParams S, const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params,
                ServedList sv, int* __restrict__ status_word)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    NetSmem& sh = *reinterpret_cast<NetSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, grp = warp >> 2, row = tid & 127;
    mlptc::load_net(sh.net, wbf, params);
    if (warp == 0) umma::tmem_alloc(&sh.tmem_base, mlptc::kTileCols * kNetGroups);
    if (tid < kNetGroups) umma::mbar_init(&sh.bar[tid], 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t d_tmem = sh.tmem_base + (uint32_t)grp * mlptc::kTileCols, a_tmem = d_tmem + mlptc::kACol;
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
    mlptc::store_constants(a_tmem + lane);
    const uint64_t n = min(*(sv.net_idx ? sv.net_count : sv.count), (unsigned long long)sv.capacity);
    const uint64_t tiles = (n + mlptc::kRows - 1) / mlptc::kRows;
    uint32_t parity = 0;
    const uint64_t stride = (uint64_t)gridDim.x * kNetGroups;
    // this thread's input row and projection residual, loaded one tile ahead
    auto load_row = [&](uint64_t t, uint4& lo, uint4& hi, float4& b) {
        const uint64_t r = t * mlptc::kRows + row;
        lo = make_uint4(0u, 0u, 0u, 0u);
        hi = lo;
        b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < tiles && r < n) {
            const uint4* xr = reinterpret_cast<const uint4*>(sv.X + r * kMlpIn);
            lo = __ldcs(xr);
            hi = __ldcs(xr + 1);
            b = __ldcs(sv.B + r);
        }
    };
    uint4 nlo, nhi;
    float4 nb;
    load_row((uint64_t)blockIdx.x * kNetGroups + grp, nlo, nhi, nb);
    bool bad = false;   // a wait of this warpgroup gave up
    for (uint64_t t = (uint64_t)blockIdx.x * kNetGroups + grp; t < tiles; t += stride) {
        const uint64_t r = t * mlptc::kRows + row;
        const float4 b = nb;
        mlptc::store_input(a_tmem + lane, nlo, nhi);
        load_row(t + stride, nlo, nhi, nb);
        // unrolled: each layer's descriptors and epilogue are fixed at compile time
#pragma unroll
        for (int l = 0; l < kMlpLayers; ++l) {
            umma::fence_before_sync();
            umma::named_sync(1 + grp, 128);
            bool timed_out = false;
            if (row == 0) {
                umma::fence_after_sync();
                mlptc::issue_layer(sh.net, l, a_tmem, d_tmem);
                umma::commit(&sh.bar[grp]);
                // one thread polls; the rest of its warp parks at __syncwarp and
                // the other warps at the named barrier, leaving the issue slots
                // to the other warpgroup's epilogue
                timed_out = !umma::mbar_wait(&sh.bar[grp], parity, mlptc::kWaitLimit);
            }
            __syncwarp();
            // the barrier also tells the warpgroup whether the wait gave up
            if (umma::named_sync_or(1 + grp, 128, timed_out)) {
                bad = true;
                break;
            }
            parity ^= 1u;
            umma::fence_after_sync();
            if (l < kMlpLayers - 1) {
                mlptc::epilogue_hidden(d_tmem + lane, a_tmem + lane);
            } else {
                float y[kMlpOut];
                mlptc::epilogue_out(d_tmem + lane, y);
                if (r < n) {
                    const uint64_t dst = sv.net_idx ? (uint64_t)__ldcs(sv.net_idx + r) : r;
                    __stcs(sv.R + dst, make_float4(b.x + y[0] * S.t_scale[0], b.y + y[1] * S.t_scale[1],
                                                   b.z + y[2] * S.t_scale[2], b.w + y[3] * S.t_scale[3]));
                }
            }
        }
        if (bad) break;
    }
    if (bad && row == 0) {
        // report, then give the MMAs in flight a second bounded wait before
        // the tensor memory is released
        atomicCAS(status_word, 0, (int)PIVBOS_ERR_DEVICE_TIMEOUT);
        umma::mbar_wait(&sh.bar[grp], parity, mlptc::kWaitLimit);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_dealloc(sh.tmem_base, mlptc::kTileCols * kNetGroups);
    }
}

// Finish: the served list in chunks of 256 consecutive entries (one round of
// the prep kernel's rays: a few neighbouring sources), each chunk deposited
// into a shared tile anchored at its first hit.
constexpr int kFinishCtasPerSm = 4;   // resident CTAs per SM (the grid is this many per SM)

template <bool EXT>
__global__ void __launch_bounds__(256, kFinishCtasPerSm)
surr_finish_kernel(const TraceParams P, const SurrParams S, ServedList sv, const float4* __restrict__ resid,
                   int64_t* __restrict__ image, int64_t* __restrict__ stats, unsigned long long* __restrict__ counter)
{
    __shared__ uint32_t tile[2 * kTileW * kTileH];   // split: 256 rays per flush, two additions per pixel each
    __shared__ unsigned long long s_item[2];
    __shared__ int w_ok[8], w_ax[8], w_ay[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const uint64_t n = min(*sv.count, (unsigned long long)sv.capacity);
    const uint64_t items = (n + 255) / 256;
    unsigned cnt[PIVBOS_RAY_NSTATUS] = {0, 0, 0, 0, 0, 0};
    // this thread's entry of an item: the straight line from the prep kernel
    // and the residual (none for a ray that never enters the box)
    struct Entry4 {
        float4 l, r;
        bool active;
    };
    auto fetch = [&](uint64_t it, Entry4& e) {
        const uint64_t pos = it * 256 + tid;
        e.active = it < items && pos < n;
        e.l = make_float4(0.f, 0.f, 0.f, 0.f);
        e.r = e.l;
        if (e.active) {
            e.l = __ldcs(sv.L + pos);
            if (!(__ldcs(sv.ids + pos) & kStraightBit)) e.r = __ldcs(resid + pos);
        }
    };
    if (tid == 0) s_item[0] = atomicAdd(counter, 1ull);
    for (int q = tid; q < 2 * kTileW * kTileH; q += blockDim.x) tile[q] = 0u;
    __syncthreads();
    int buf = 0;
    uint64_t it = s_item[0];
    Entry4 cur;
    fetch(it, cur);
    // Three barriers per item: the anchors (and the next item) are known, the
    // deposits are in the tile, the tile is flushed and clear again.  The
    // next item's entries load while this one deposits.
    while (it < items) {
        if (tid == 0) s_item[buf ^ 1] = atomicAdd(counter, 1ull);
        RayOut r;
        r.status = PIVBOS_RAY_MISS;
        int fx = 0, fy = 0;
        if (cur.active) {
            const float res[4] = {cur.r.x, cur.r.y, cur.r.z, cur.r.w};
            r.status = PIVBOS_RAY_REACHED;
            surr_sensor<EXT>(P.o, S, cur.l.x, cur.l.y, cur.l.z, cur.l.w, res, r.status, r.px, r.py);
            r.w = 1.0f;
            if constexpr (EXT) {
                // the ray's radiance from its direction at the source: the
                // straight line's slopes
                if (P.o.rad_mode) {
                    const float inn = rsqrtf(fmaf(cur.l.z, cur.l.z, fmaf(cur.l.w, cur.l.w, 1.0f)));
                    r.w = ray_radiance(P.o, cur.l.z * inn, cur.l.w * inn, inn);
                }
            }
            cnt[r.status]++;
            if (r.status == PIVBOS_RAY_REACHED) {
                float f;
                fx = df_floor(r.px, f) - kTileW / 2;
                fy = df_floor(r.py, f) - kTileH / 2;
            }
        }
        // the tile's anchor: the first ray that reaches the sensor, in thread order
        const bool reached = cur.active && r.status == PIVBOS_RAY_REACHED;
        const unsigned dep = __ballot_sync(0xffffffffu, reached);
        const int leader = dep ? __ffs(dep) - 1 : 0;
        const int lx = __shfl_sync(0xffffffffu, fx, leader), ly = __shfl_sync(0xffffffffu, fy, leader);
        if (lane == 0) {
            w_ok[warp] = dep != 0;
            w_ax[warp] = lx;
            w_ay[warp] = ly;
        }
        __syncthreads();
        int ax = -(1 << 28), ay = -(1 << 28);
        for (int w = 0; w < nw; ++w)
            if (w_ok[w]) {
                ax = w_ax[w];
                ay = w_ay[w];
                break;
            }
        const uint64_t it_next = s_item[buf ^ 1];
        Entry4 nxt;
        fetch(it_next, nxt);
        if (reached) deposit_ray<EXT>(P.o, r.px, r.py, tile, ax, ay, image, r.w, dep);
        __syncthreads();
        for (int q = tid; q < kTileW * kTileH; q += blockDim.x) {
            const unsigned long long v = take_split(tile, q);
            if (v) {
                const int gx = ax + (q % kTileW), gy = ay + (q / kTileW);
                atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * P.o.W + gx]), v);
            }
        }
        __syncthreads();
        it = it_next;
        cur = nxt;
        buf ^= 1;
    }
    if (stats) {
#pragma unroll
        for (int q = 0; q < PIVBOS_RAY_NSTATUS; ++q)
            if (cnt[q]) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[q]), (unsigned long long)cnt[q]);
    }
}

// Direct render, for a surrogate whose served bins all take the projection
// alone: the prep and finish kernels' work in one pass, with no served list
// in HBM.  Items of kMaxOrderRays consecutive rays of the Morton-ordered
// (slot, ray) space (one source or a few neighbouring ones); each ray is
// generated, served by the projection (or, never entering the box, by its
// straight line) and deposited into the CTA's split tile, anchored at the
// round's first hit (a round is 256 rays, one per thread) and flushed after
// every round; rays of bins without a predictor go to the fallback list (a
// warp-level append).  Two barriers per round: the anchors are known, the
// deposits are in the tile (the flush then runs while the next round's rays
// are prepared).
// The deposits are the finish kernel's quanta for the same rays, so the
// image and status counts are the three-kernel path's, bit for bit.
constexpr int kDirectCtasPerSm = 4;

template <bool EXT>
__global__ void __launch_bounds__(256, kDirectCtasPerSm)
surr_direct_kernel(const TraceParams P, const SurrParams S, uint64_t c0, uint64_t c1,
                   uint32_t* __restrict__ fb_ids, unsigned long long* __restrict__ fb_count, uint32_t fb_capacity,
                   int64_t* __restrict__ image, int64_t* __restrict__ stats)
{
    __shared__ uint32_t tile[2 * kTileW * kTileH];   // split: 256 rays per flush, two additions per pixel each
    __shared__ uint32_t order[kMaxOrderRays];
    __shared__ int w_ok[8], w_ax[8], w_ay[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const uint32_t rps = P.rays_per_source;
    unsigned cnt[PIVBOS_RAY_NSTATUS] = {0, 0, 0, 0, 0, 0};
    for (int q = tid; q < 2 * kTileW * kTileH; q += blockDim.x) tile[q] = 0u;
    const uint64_t items = (c1 - c0 + kMaxOrderRays - 1) / kMaxOrderRays;
    for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint64_t first = c0 + it * kMaxOrderRays;
        const uint32_t n_here = (uint32_t)(min(first + kMaxOrderRays, c1) - first);
        const bool reorder = P.reorder && S.born_k >= 8;
        if (reorder) order_chunk(P, order, first, n_here);
        for (uint32_t r0 = 0; r0 < n_here; r0 += 256) {
            const uint32_t pos = r0 + tid;
            const bool active = pos < n_here;
            const uint64_t idx = first + (reorder && active ? (order[pos] & 0x7ffu) : pos);
            int mode = 3;   // 0 projection, 1 fallback, 2 straight, 3 none
            RayOut r;
            r.status = PIVBOS_RAY_MISS;
            r.w = 1.0f;
            if (active) {
                const uint32_t flat = (uint32_t)idx;
                const uint32_t slot = flat / rps, k = flat - slot * rps;
                const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
                const float2* sp = P.src_df + 3 * (size_t)slot;
                const float2 a = __ldg(sp), b = __ldg(sp + 1), c = __ldg(sp + 2);
                Entry e;
                surr_entry_f(P, S, a.x + a.y, b.x + b.y, c.x + c.y, sid, k, e);
                if (!e.enters) mode = 2;
                else mode = ((__ldg(S.bin_ok + (e.bin >> 5)) >> (e.bin & 31)) & 1u) ? 0 : 1;
                if (mode != 1) {
                    float res[4] = {0.f, 0.f, 0.f, 0.f};
                    if (mode == 0) born_residual(S, e, res);
                    r.status = PIVBOS_RAY_REACHED;
                    surr_sensor<EXT>(P.o, S, e.xs, e.ys, e.ux, e.uy, res, r.status, r.px, r.py);
                    if constexpr (EXT) {
                        // the ray's radiance from its direction at the source
                        if (P.o.rad_mode) {
                            const float inn = rsqrtf(fmaf(e.ux, e.ux, fmaf(e.uy, e.uy, 1.0f)));
                            r.w = ray_radiance(P.o, e.ux * inn, e.uy * inn, inn);
                        }
                    }
                    cnt[r.status]++;
                }
            }
            // the fallback list: one atomic per warp
            const unsigned fbm = __ballot_sync(0xffffffffu, mode == 1);
            if (fbm) {
                unsigned long long fb0 = 0ull;
                if (lane == __ffs(fbm) - 1) fb0 = atomicAdd(fb_count, (unsigned long long)__popc(fbm));
                fb0 = __shfl_sync(0xffffffffu, fb0, __ffs(fbm) - 1);
                if (mode == 1) {
                    const unsigned long long q = fb0 + __popc(fbm & ((1u << lane) - 1u));
                    if (q < fb_capacity) fb_ids[q] = (uint32_t)idx;
                    else atomicCAS(P.status_word, 0, (int)PIVBOS_ERR_OVERFLOW);   // cannot happen: capacity = rays
                }
            }
            // the tile's anchor: the round's first hit in thread order
            const bool reached = mode != 1 && r.status == PIVBOS_RAY_REACHED;
            int fx = 0, fy = 0;
            if (reached) {
                float f;
                fx = df_floor(r.px, f) - kTileW / 2;
                fy = df_floor(r.py, f) - kTileH / 2;
            }
            const unsigned dep = __ballot_sync(0xffffffffu, reached);
            const int leader = dep ? __ffs(dep) - 1 : 0;
            const int lx = __shfl_sync(0xffffffffu, fx, leader), ly = __shfl_sync(0xffffffffu, fy, leader);
            if (lane == 0) {
                w_ok[warp] = dep != 0;
                w_ax[warp] = lx;
                w_ay[warp] = ly;
            }
            __syncthreads();
            int ax = -(1 << 28), ay = -(1 << 28);
            for (int w = 0; w < nw; ++w)
                if (w_ok[w]) {
                    ax = w_ax[w];
                    ay = w_ay[w];
                    break;
                }
            if (reached) deposit_ray<EXT>(P.o, r.px, r.py, tile, ax, ay, image, r.w, dep);
            __syncthreads();
            for (int q = tid; q < kTileW * kTileH; q += blockDim.x) {
                const unsigned long long v = take_split(tile, q);
                if (v) {
                    const int gx = ax + (q % kTileW), gy = ay + (q / kTileW);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * P.o.W + gx]), v);
                }
            }
        }
    }
    if (stats) {
#pragma unroll
        for (int q = 0; q < PIVBOS_RAY_NSTATUS; ++q) {
            unsigned v = cnt[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[q]), (unsigned long long)v);
        }
    }
}

// Per-ray surrogate sensor positions for checking (flag 0 surrogate, 1 plain
// fallback (traced here), 2 never enters the box (straight)).
template <int INTEG>
__global__ void surr_sensor_kernel(const TraceParams P, const SurrParams S, const float* __restrict__ Y,
                                   const int64_t* __restrict__ ids, int64_t n, double* __restrict__ out_px,
                                   int* __restrict__ out_flag, int* __restrict__ out_status)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t sid, k;
    df sx, sy, sz;
    Entry e;
    surr_ray_by_id(P, S, (uint64_t)ids[q], sid, k, sx, sy, sz, e);
    // 0: the network's corrected projection, 3: the projection alone, 1: the
    // plain fallback, 2: never enters the box
    int flag = !e.enters ? 2 : (((S.bin_ok[e.bin >> 5] >> (e.bin & 31)) & 1u) ? 0 : 1);
    if (flag == 0 && !net_bin(S, e.bin)) flag = 3;
    int status = PIVBOS_RAY_REACHED;
    df px = dfv(0.f), py = dfv(0.f);
    if (flag == 1) {
        RayOut r;
        trace_ray<INTEG, false>(P, sx, sy, sz, sid + P.source_offset, k, r, nullptr);
        status = r.status;
        px = r.px;
        py = r.py;
    } else {
        // the straight line (a ray that never enters the box) or the
        // surrogate's exit line, as the render's finish kernel takes them
        float res[4] = {0.f, 0.f, 0.f, 0.f};
        if (flag == 0 || flag == 3) {
            float born[4];
            born_residual(S, e, born);
            surr_residual(S, born, Y + q * 4, flag == 0, res);
        }
        surr_sensor(P.o, S, e.xs, e.ys, e.ux, e.uy, res, status, px, py);
    }
    out_px[2 * q] = df_to_double(px);
    out_px[2 * q + 1] = df_to_double(py);
    out_flag[q] = flag;
    out_status[q] = status;
}

// Encoded features of given rays (the network input of surr_sensor_kernel).
__global__ void surr_features_kernel(const TraceParams P, const SurrParams S, const int64_t* __restrict__ ids,
                                     int64_t n, __nv_bfloat16* __restrict__ X)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t sid, k;
    df sx, sy, sz;
    Entry e;
    surr_ray_by_id(P, S, (uint64_t)ids[q], sid, k, sx, sy, sz, e);
    float born[4];
    born_residual(S, e, born);
    encode_features(S, e.f, born, X + (size_t)q * kMlpIn);
}

}  // namespace pivbos

