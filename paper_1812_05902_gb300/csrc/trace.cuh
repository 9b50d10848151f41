// Device functions of the ray tracer: one GPU thread follows one ray through
// all four steps of the method (arXiv 1812.05902, Sec. 3 and Sec. 3.5).
//
// Precision plan.  GB300 issues FP64 at 1/64 of its FP32 rate, so the
// tracer uses no FP64 arithmetic on its hot path:
//  * positions and directions outside the density box, the lens surfaces
//    and the sensor plane are double-float (df64.cuh, ~48 bits): the sensor
//    position must be right to 1e-5 pixel (1.7e-10 m at 17 um pitch) on
//    coordinates up to ~1e-2 m, beyond FP32's 24 bits;
//  * decisions (apertures, clear radii, hemisphere, total internal
//    reflection) compare the FP32 leading parts;
//  * the lens point is drawn from 53-bit uniforms: the radius a sqrt(u1) and
//    the angle 2 pi u2 (df_sincospi) in double-float;
//  * integration: the ray is carried as a straight reference line
//    R0 + T0 t (double-float) plus an FP32 perturbation (rho, tau) that the
//    Runge-Kutta update acts on.  The update of Eq. 3 is linear in (R, T), so
//    R_i = R0 + T0 t_i + rho_i, T_i = T0 + tau_i gives exactly
//        rho_{i+1} = rho_i + [tau_i + (A + 2B)/6] dt,
//        tau_{i+1} = tau_i + (A + 4B + C)/6,
//    and FP32 rounding applies to the deflection (~1e-5 rad, ~1e-5 m), not
//    to absolute positions (~1 m) and directions (~1);
//  * the reference line is stepped in double-float grid coordinates and a
//    sample's cell fraction is taken as (hi - cell) + (lo + offset), so the
//    field is evaluated where the oracle evaluates it to ~1e-7 of a cell.
#pragma once

#include <math.h>

#include "common.cuh"
#include "df64.cuh"

namespace pivbos {

__device__ __forceinline__ df dfk(dfc c) { return df{c.hi, c.lo}; }

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Only the first two
// output words are used (the lens point needs two uniforms, Sec. 3.1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_lens_words(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                  uint64_t k0, uint64_t k1,
                                                  uint64_t& w0, uint64_t& w1)
{
    const uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
    const uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(kM0, c0), lo0 = kM0 * c0;
        const uint64_t hi1 = __umul64hi(kM1, c2), lo1 = kM1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += kW0; k1 += kW1;
    }
    w0 = c0;
    w1 = c1;
}

// 53-bit uniform ((w >> 11) + 1/2) 2^-53 as a double-float: the top 24 bits
// exactly in hi, the remaining 29 bits (and the half) in lo.
__device__ __forceinline__ df u01_df(uint64_t w)
{
    const uint64_t m = w >> 11;
    const float hi = (float)(uint32_t)(m >> 29) * 0x1p-24f;
    const float lo = ((float)(uint32_t)(m & 0x1fffffffull) + 0.5f) * 0x1p-53f;
    return fast_two_sum(hi, lo);
}

// ---------------------------------------------------------------------------
// Trilinear sample of the float4 node field at grid coordinates (clamped).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t)
{
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y),
                       fmaf(t, b.z - a.z, a.z), fmaf(t, b.w - a.w, a.w));
}

__device__ __forceinline__ float4 sample_field(const DevMedium& m, float gx, float gy, float gz)
{
    gx = fminf(fmaxf(gx, 0.0f), (float)(m.n[0] - 1));
    gy = fminf(fmaxf(gy, 0.0f), (float)(m.n[1] - 1));
    gz = fminf(fmaxf(gz, 0.0f), (float)(m.n[2] - 1));
    const int i = min((int)gx, m.n[0] - 2);
    const int j = min((int)gy, m.n[1] - 2);
    const int k = min((int)gz, m.n[2] - 2);
    const float fx = gx - (float)i, fy = gy - (float)j, fz = gz - (float)k;
    const int sy = m.n[0];
    const int sz = m.n[0] * m.n[1];
    const float4* p = m.field + ((k * m.n[1] + j) * m.n[0] + i);
    const float4 c000 = __ldg(p), c100 = __ldg(p + 1);
    const float4 c010 = __ldg(p + sy), c110 = __ldg(p + sy + 1);
    const float4 c001 = __ldg(p + sz), c101 = __ldg(p + sz + 1);
    const float4 c011 = __ldg(p + sz + sy), c111 = __ldg(p + sz + sy + 1);
    const float4 x00 = lerp4(c000, c100, fx), x10 = lerp4(c010, c110, fx);
    const float4 x01 = lerp4(c001, c101, fx), x11 = lerp4(c011, c111, fx);
    const float4 y0 = lerp4(x00, x10, fy), y1 = lerp4(x01, x11, fy);
    return lerp4(y0, y1, fz);
}

// Eq. 6: D = n grad n, from the sampled n - 1 and gradient.
__device__ __forceinline__ float3 eval_D(const DevMedium& m, float gx, float gy, float gz)
{
    const float4 v = sample_field(m, gx, gy, gz);
    const float n = 1.0f + v.x;
    return make_float3(n * v.y, n * v.z, n * v.w);
}

// Cell index and fraction of the grid coordinate gh + gl along one axis of
// N nodes, clamped to [0, N-1].  gh is the leading part of a double-float
// coordinate (up to N-1 cells) and gl the small rest (its low part plus the
// FP32 offset of the sample point), so the fraction keeps ~1e-7 of a cell
// wherever the point is in the grid.
__device__ __forceinline__ void cell_split(float gh, float gl, int N, int& i, float& f)
{
    // Branch-free: below the grid (or NaN) the cell is 0 and the fraction
    // saturates to 0, above it the cell is N-2 and the fraction saturates to 1.
    const float s = gh + gl;
    i = min(max((int)s, 0), N - 2);
    f = __saturatef(__fadd_rn(__fsub_rn(gh, (float)i), gl));
}

// Corners of the last cell a ray sampled.  Consecutive Runge-Kutta stages
// and steps mostly fall in the same cell (the first stage of a step lies
// within ~1e-11 m of the last stage of the previous one), so keeping the
// eight float4 corners in registers saves most of the gathers.
template <bool CACHE>
struct CellCache {
    __device__ __forceinline__ void reset() {}
};
template <>
struct CellCache<true> {
    int cell;
    float4 c[8];
    __device__ __forceinline__ void reset() { cell = -1; }
};

// D = n grad n (Eq. 6) from the trilinear samples of n - 1 and grad n at the
// grid point gh + gl (see cell_split), written as the weighted sum of the
// eight corner values, w = (1-fx or fx)(1-fy or fy)(1-fz or fz).  The fourth
// component is the sampled n - 1 (for the optical path; unused otherwise).
template <bool CACHE>
__device__ __forceinline__ float4 eval_D_split(const DevMedium& m, CellCache<CACHE>& cc, float hx, float lx, float hy,
                                               float ly, float hz, float lz)
{
    int i, j, k;
    float fx, fy, fz;
    cell_split(hx, lx, m.n[0], i, fx);
    cell_split(hy, ly, m.n[1], j, fy);
    cell_split(hz, lz, m.n[2], k, fz);
    const int cell = (k * m.n[1] + j) * m.n[0] + i;
    float4 c[8];
    if constexpr (CACHE) {
        if (cell != cc.cell) {
            const int sy = m.n[0];
            const int sz = m.n[0] * m.n[1];
            const float4* p = m.field + cell;
            cc.c[0] = __ldg(p);           cc.c[1] = __ldg(p + 1);
            cc.c[2] = __ldg(p + sy);      cc.c[3] = __ldg(p + sy + 1);
            cc.c[4] = __ldg(p + sz);      cc.c[5] = __ldg(p + sz + 1);
            cc.c[6] = __ldg(p + sz + sy); cc.c[7] = __ldg(p + sz + sy + 1);
            cc.cell = cell;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = cc.c[q];
    } else {
        const int sy = m.n[0];
        const int sz = m.n[0] * m.n[1];
        const float4* p = m.field + cell;
        c[0] = __ldg(p);           c[1] = __ldg(p + 1);
        c[2] = __ldg(p + sy);      c[3] = __ldg(p + sy + 1);
        c[4] = __ldg(p + sz);      c[5] = __ldg(p + sz + 1);
        c[6] = __ldg(p + sz + sy); c[7] = __ldg(p + sz + sy + 1);
    }
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w00 = gy * gz, w10 = fy * gz, w01 = gy * fz, w11 = fy * fz;
    const float w[8] = {gx * w00, fx * w00, gx * w10, fx * w10, gx * w01, fx * w01, gx * w11, fx * w11};
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        v.x = fmaf(w[q], c[q].x, v.x);
        v.y = fmaf(w[q], c[q].y, v.y);
        v.z = fmaf(w[q], c[q].z, v.z);
        v.w = fmaf(w[q], c[q].w, v.w);
    }
    const float n = 1.0f + v.x;
    return make_float4(n * v.y, n * v.z, n * v.w, v.x);
}

struct RayOut {
    df px, py;     // sensor pixel coordinates
    int status;
    int steps;
    float w;       // radiance weight (Sec. 3.1; 1 without a Mie radiance)
};

// Sec. 3.1: the radiance of a ray leaving its source along d0 (unit), from
// the optics' Mie table: theta = acos(d0.L) from the laser direction L,
// |S1|^2 and |S2|^2 interpolated linearly in theta (the table is already
// divided by its maximum); unpolarised light takes their mean, a laser
// polarised along p takes |S2|^2 cos^2(phi) + |S1|^2 sin^2(phi), phi the
// angle between p and the scattering plane (which holds L and d0).
__device__ __forceinline__ float ray_radiance(const DevOptics& o, float dx, float dy, float dz)
{
    const float c = fminf(fmaxf(fmaf(dx, o.rad_L[0], fmaf(dy, o.rad_L[1], dz * o.rad_L[2])), -1.0f), 1.0f);
    const float t = acosf(c) * (0.31830988618379067f * (float)(o.rad_n - 1));
    const int i = min((int)t, o.rad_n - 2);
    const float f = t - (float)i;
    const float2 a = __ldg(o.rad + i), b = __ldg(o.rad + i + 1);
    const float s1 = fmaf(f, b.x - a.x, a.x), s2 = fmaf(f, b.y - a.y, a.y);
    if (o.rad_mode != 2) return 0.5f * (s1 + s2);
    const float ex = fmaf(-c, o.rad_L[0], dx), ey = fmaf(-c, o.rad_L[1], dy), ez = fmaf(-c, o.rad_L[2], dz);
    const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float pe = fmaf(o.rad_pol[0], ex, fmaf(o.rad_pol[1], ey, o.rad_pol[2] * ez));
    const float c2 = e2 > 0.0f ? pe * pe / e2 : 0.5f;
    return fmaf(s2 - s1, c2, s1);
}

__device__ __forceinline__ void put3(double* dst, df x, df y, df z)
{
    dst[0] = df_to_double(x);
    dst[1] = df_to_double(y);
    dst[2] = df_to_double(z);
}

// Sec. 3.1: the ray from source (sx, sy, sz) to its lens point, unit direction.
__device__ __forceinline__ void ray_start(const TraceParams& P, df sx, df sy, df sz, uint32_t sid, uint32_t rid,
                                          df& dx, df& dy, df& dz)
{
    const DevOptics& o = P.o;
    uint64_t w0, w1;
    philox_lens_words(rid, sid, P.frame, 0ull, P.seed, 0ull, w0, w1);
    const df rr = df_mul(dfk(o.aim_r), df_sqrt(u01_df(w0)));
    const df u2 = u01_df(w1);
    df sn, cs;
    df_sincospi(df{2.0f * u2.hi, 2.0f * u2.lo}, sn, cs);
    dx = df_sub(df_mul(rr, cs), sx);
    dy = df_sub(df_mul(rr, sn), sy);
    dz = df_sub(dfk(o.aim_z), sz);
    const df inv = df_rsqrt(df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz)));
    dx = df_mul(dx, inv);
    dy = df_mul(dy, inv);
    dz = df_mul(dz, inv);
}

// Whether the straight ray R + t d (t >= 0) enters the density box, and the
// parameter tn of the entry point (0 for a start inside the box).  An FP32
// slab test decides whether and through which face; the entry parameter of
// that face is then solved in double-float, so integration starts on the
// face (a start shifted along the ray would shift every field sample).
__device__ __forceinline__ bool box_entry(const DevMedium& m, df Rx, df Ry, df Rz, df dx, df dy, df dz, df& tn)
{
    tn = dfv(0.0f);
    const df lo0 = dfk(m.lo[0]), lo1 = dfk(m.lo[1]), lo2 = dfk(m.lo[2]);
    const df hi0 = dfk(m.hi[0]), hi1 = dfk(m.hi[1]), hi2 = dfk(m.hi[2]);
    if (!df_lt(Rx, lo0) && !df_gt(Rx, hi0) && !df_lt(Ry, lo1) && !df_gt(Ry, hi1) && !df_lt(Rz, lo2) &&
        !df_gt(Rz, hi2))
        return true;
    float t_near = -INFINITY, t_far = INFINITY;
    int a_near = -1;
    bool ok = true;
    const float dd[3] = {dx.hi, dy.hi, dz.hi};
    const float RR[3] = {Rx.hi, Ry.hi, Rz.hi};
    const float LO[3] = {m.lo[0].hi, m.lo[1].hi, m.lo[2].hi};
    const float HI[3] = {m.hi[0].hi, m.hi[1].hi, m.hi[2].hi};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0f) {
            if (RR[a] < LO[a] || RR[a] > HI[a]) ok = false;
        } else {
            const float inv = 1.0f / dd[a];
            const float t1 = (LO[a] - RR[a]) * inv;
            const float t2 = (HI[a] - RR[a]) * inv;
            const float tmin = fminf(t1, t2);
            if (tmin > t_near) {
                t_near = tmin;
                a_near = a;
            }
            t_far = fminf(t_far, fmaxf(t1, t2));
        }
    }
    if (!(ok && t_near <= t_far && t_near >= 0.0f && a_near >= 0)) return false;
    const df Ra = a_near == 0 ? Rx : (a_near == 1 ? Ry : Rz);
    const df da = a_near == 0 ? dx : (a_near == 1 ? dy : dz);
    const dfc face = da.hi > 0.0f ? m.lo[a_near] : m.hi[a_near];
    tn = df_div(df_sub(dfk(face), Ra), da);
    if (tn.hi < 0.0f) tn = dfv(0.0f);
    return true;
}

// Sec. 3.3 and 3.4: from a point and direction in object space through the
// optical elements to the sensor plane.  Leaves status unchanged if the ray
// reaches the sensor array; (R, d) end as the state at the sensor.
//
// Written once over a number type: N = DfOps (double-float, the exact
// path) or F32Ops (FP32, for the surrogate's approximate exit lines, whose
// error budget is a thousand times looser); DfOps maps every operation onto
// the double-float function it names.
struct DfOps {
    using T = df;
    static __device__ __forceinline__ T k(dfc c) { return dfk(c); }
    static __device__ __forceinline__ T v(float a) { return dfv(a); }
    static __device__ __forceinline__ float hi(T a) { return a.hi; }
    static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return df_sub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return df_fma(a, b, c); }
    static __device__ __forceinline__ T sqr(T a) { return df_sqr(a); }
    static __device__ __forceinline__ T sqrt(T a) { return df_sqrt(a); }
    static __device__ __forceinline__ T div(T a, T b) { return df_div(a, b); }
    static __device__ __forceinline__ T rcp(T a) { return df_rcp(a); }
    static __device__ __forceinline__ T rsqrt(T a) { return df_rsqrt(a); }
    static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
    static __device__ __forceinline__ T add_f(T a, float b) { return df_add_f(a, b); }
    static __device__ __forceinline__ bool lt(T a, T b) { return df_lt(a, b); }
    static __device__ __forceinline__ int floor_i(T a) { float f; return df_floor(a, f); }
};
struct F32Ops {
    using T = float;
    static __device__ __forceinline__ T k(dfc c) { return c.hi + c.lo; }
    static __device__ __forceinline__ T v(float a) { return a; }
    static __device__ __forceinline__ float hi(T a) { return a; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ T sqr(T a) { return a * a; }
    static __device__ __forceinline__ T sqrt(T a) { return sqrtf(a); }
    static __device__ __forceinline__ T div(T a, T b) { return a / b; }
    static __device__ __forceinline__ T rcp(T a) { return 1.0f / a; }
    static __device__ __forceinline__ T rsqrt(T a) { return rsqrtf(a); }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T add_f(T a, float b) { return a + b; }
    static __device__ __forceinline__ bool lt(T a, T b) { return a < b; }
    static __device__ __forceinline__ int floor_i(T a) { return (int)floorf(a); }
};

// EXT = false compiles the plain elements only (spheres, planes, ideal thin
// lenses, stops) and a sensor square to the axis; EXT = true adds mirrors,
// lens arrays and a turned sensor.  Launchers pick EXT = false unless the
// optics hold one of those, so the plain path's code stays as compact as
// before they existed.
template <class N = DfOps, bool EXT = true>
__device__ __forceinline__ void optics_to_sensor(const DevOptics& o, typename N::T& Rx, typename N::T& Ry,
                                                 typename N::T& Rz, typename N::T& dx, typename N::T& dy,
                                                 typename N::T& dz, int& status, typename N::T& px,
                                                 typename N::T& py)
{
    using T = typename N::T;
    for (int s = 0; s < o.ns && status == PIVBOS_RAY_REACHED; ++s) {
        const DevSurface& S = o.s[s];
        if (!(N::hi(dz) > 0.0f)) { status = PIVBOS_RAY_MISS; break; }
        const T inv_dz = N::rcp(dz);
        const T t0 = N::mul(N::sub(N::k(S.z), Rz), inv_dz);
        if ((S.type == PIVBOS_SURF_SPHERE || (EXT && S.type == PIVBOS_SURF_MIRROR)) && S.R_f != 0.0f) {
            // vertex-relative quadratic t^2 + 2 b t + c = 0 from the point Q
            // on the vertex plane; the vertex-side root has the smaller
            // magnitude: t = c / (-b - sign(b) sqrt(b^2 - c))
            const T Qx = N::fma(t0, dx, Rx), Qy = N::fma(t0, dy, Ry);
            const T R = N::k(S.R);
            const T b = N::sub(N::add(N::mul(dx, Qx), N::mul(dy, Qy)), N::mul(R, dz));
            const T c = N::add(N::sqr(Qx), N::sqr(Qy));
            const T disc = N::sub(N::sqr(b), c);
            if (N::hi(disc) < 0.0f) { status = PIVBOS_RAY_MISS; break; }
            const T sq = N::sqrt(disc);
            const T den = N::hi(b) >= 0.0f ? N::sub(N::neg(b), sq) : N::add(N::neg(b), sq);
            const T t1 = N::hi(den) != 0.0f ? N::div(c, den) : N::v(0.0f);
            if (N::hi(N::add(t0, t1)) < 0.0f) { status = PIVBOS_RAY_MISS; break; }
            const T Hx = N::fma(t1, dx, Qx), Hy = N::fma(t1, dy, Qy), Hz = N::mul(t1, dz);
            const T HzR = N::sub(Hz, R);
            if (!(N::hi(HzR) * S.R_f < 0.0f)) { status = PIVBOS_RAY_MISS; break; }
            if (N::hi(Hx) * N::hi(Hx) + N::hi(Hy) * N::hi(Hy) > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
            const T invR = N::k(S.invR);
            T Nx = N::mul(Hx, invR), Ny = N::mul(Hy, invR), Nz = N::mul(HzR, invR);
            if (N::hi(Nx) * N::hi(dx) + N::hi(Ny) * N::hi(dy) + N::hi(Nz) * N::hi(dz) > 0.0f) {
                Nx = N::neg(Nx); Ny = N::neg(Ny); Nz = N::neg(Nz);
            }
            if (EXT && S.type == PIVBOS_SURF_MIRROR) {
                // Sec. 3.3, item 1: d' = d - 2 (d.N) N; then unfold about the
                // vertex plane (z - z_v -> z_v - z, d_z -> -d_z)
                const T dn2 = N::mul(N::v(2.0f), N::add(N::add(N::mul(Nx, dx), N::mul(Ny, dy)), N::mul(Nz, dz)));
                dx = N::sub(dx, N::mul(dn2, Nx));
                dy = N::sub(dy, N::mul(dn2, Ny));
                dz = N::neg(N::sub(dz, N::mul(dn2, Nz)));
                Rx = Hx;
                Ry = Hy;
                Rz = N::sub(N::k(S.z), Hz);
                continue;
            }
            // Eq. 7, vector form
            const T eta = N::k(S.eta);
            const T ci = N::neg(N::add(N::add(N::mul(Nx, dx), N::mul(Ny, dy)), N::mul(Nz, dz)));
            const T kk = N::sub(N::v(1.0f), N::mul(N::k(S.eta2), N::sub(N::v(1.0f), N::sqr(ci))));
            if (N::hi(kk) < 0.0f) { status = PIVBOS_RAY_TIR; break; }
            const T a = N::sub(N::mul(eta, ci), N::sqrt(kk));
            dx = N::fma(eta, dx, N::mul(a, Nx));
            dy = N::fma(eta, dy, N::mul(a, Ny));
            dz = N::fma(eta, dz, N::mul(a, Nz));
            Rx = Hx;
            Ry = Hy;
            Rz = N::add(N::k(S.z), Hz);
        } else {
            if (N::hi(t0) < 0.0f) { status = PIVBOS_RAY_MISS; break; }
            Rx = N::fma(t0, dx, Rx);
            Ry = N::fma(t0, dy, Ry);
            Rz = N::k(S.z);
            const float r2 = N::hi(Rx) * N::hi(Rx) + N::hi(Ry) * N::hi(Ry);
            if (S.type == PIVBOS_SURF_STOP) {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_STOP; break; }
            } else if (EXT && S.type == PIVBOS_SURF_MIRROR) {
                // flat mirror square to the axis: reflection and unfolding
                // about its own plane leave the ray as it was
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
            } else if (S.type == PIVBOS_SURF_IDEAL_THIN || (EXT && S.type == PIVBOS_SURF_LENS_ARRAY)) {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
                const T invf = N::k(S.inv_f);
                // position relative to the lens centre: the lenslet of the
                // ray's cell for an array (centres at multiples of the pitch)
                T xr = Rx, yr = Ry;
                if (EXT && S.type == PIVBOS_SURF_LENS_ARRAY) {
                    const T p = N::k(S.R), ip = N::k(S.invR);
                    const float ci = (float)N::floor_i(N::add_f(N::mul(Rx, ip), 0.5f));
                    const float cj = (float)N::floor_i(N::add_f(N::mul(Ry, ip), 0.5f));
                    xr = N::sub(Rx, N::mul(p, N::v(ci)));
                    yr = N::sub(Ry, N::mul(p, N::v(cj)));
                }
                const T ux = N::sub(N::mul(dx, inv_dz), N::mul(xr, invf));
                const T uy = N::sub(N::mul(dy, inv_dz), N::mul(yr, invf));
                const T inn = N::rsqrt(N::add_f(N::add(N::sqr(ux), N::sqr(uy)), 1.0f));
                dx = N::mul(ux, inn);
                dy = N::mul(uy, inn);
                dz = inn;
            } else {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
                // flat surface, normal (0, 0, -1)
                const T eta = N::k(S.eta);
                const T kk = N::sub(N::v(1.0f), N::mul(N::k(S.eta2), N::sub(N::v(1.0f), N::sqr(dz))));
                if (N::hi(kk) < 0.0f) { status = PIVBOS_RAY_TIR; break; }
                const T a = N::sub(N::mul(eta, dz), N::sqrt(kk));
                dx = N::mul(eta, dx);
                dy = N::mul(eta, dy);
                dz = N::sub(N::mul(eta, dz), a);
            }
        }
    }

    // ---- Sec. 3.4: sensor plane -------------------------------------------
    px = N::v(0.0f);
    py = N::v(0.0f);
    bool turned = false;
    if constexpr (EXT) turned = o.tilted != 0;
    if (EXT && turned && status == PIVBOS_RAY_REACHED) {
        // a turned sensor: the plane through (0, 0, sensor_z) with normal en,
        // pixel axes eu, ev
        const T enx = N::k(o.en[0]), eny = N::k(o.en[1]), enz = N::k(o.en[2]);
        const T dn = N::add(N::add(N::mul(dx, enx), N::mul(dy, eny)), N::mul(dz, enz));
        const T cz = N::sub(N::k(o.sensor_z), Rz);
        const T t = N::div(N::sub(N::mul(cz, enz), N::add(N::mul(Rx, enx), N::mul(Ry, eny))), dn);
        if (!(N::hi(dn) > 0.0f) || N::hi(t) < 0.0f) {
            status = PIVBOS_RAY_MISS;
        } else {
            const T Xx = N::fma(t, dx, Rx), Xy = N::fma(t, dy, Ry), Xz = N::sub(N::mul(t, dz), cz);
            const T ipitch = N::k(o.inv_pitch);
            const T u = N::add(N::add(N::mul(Xx, N::k(o.eu[0])), N::mul(Xy, N::k(o.eu[1]))), N::mul(Xz, N::k(o.eu[2])));
            const T w = N::add(N::add(N::mul(Xx, N::k(o.ev[0])), N::mul(Xy, N::k(o.ev[1]))), N::mul(Xz, N::k(o.ev[2])));
            px = N::add_f(N::mul(u, ipitch), o.half_w);
            py = N::add_f(N::mul(w, ipitch), o.half_h);
            const bool inx = !N::lt(px, N::v(0.0f)) && N::lt(px, N::v((float)o.W));
            const bool iny = !N::lt(py, N::v(0.0f)) && N::lt(py, N::v((float)o.H));
            if (!(inx && iny)) status = PIVBOS_RAY_OFF_SENSOR;
        }
    } else if (status == PIVBOS_RAY_REACHED) {
        if (!(N::hi(dz) > 0.0f)) {
            status = PIVBOS_RAY_MISS;
        } else {
            const T t = N::mul(N::sub(N::k(o.sensor_z), Rz), N::rcp(dz));
            if (N::hi(t) < 0.0f) {
                status = PIVBOS_RAY_MISS;
            } else {
                const T ipitch = N::k(o.inv_pitch);
                px = N::add_f(N::mul(N::fma(t, dx, Rx), ipitch), o.half_w);
                py = N::add_f(N::mul(N::fma(t, dy, Ry), ipitch), o.half_h);
                const bool inx = !N::lt(px, N::v(0.0f)) && N::lt(px, N::v((float)o.W));
                const bool iny = !N::lt(py, N::v(0.0f)) && N::lt(py, N::v((float)o.H));
                if (!(inx && iny)) status = PIVBOS_RAY_OFF_SENSOR;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One ray through all stages.  INTEG: PIVBOS_EULER or PIVBOS_RK4.  If st is
// not null the full exit state is written (parity path).
// ---------------------------------------------------------------------------
template <int INTEG, bool CACHE, bool EXT = true>
__device__ __forceinline__ void trace_ray(const TraceParams& P, df sx, df sy, df sz, uint32_t sid, uint32_t rid,
                                          RayOut& out, pivbos_ray_state* st)
{
    const DevMedium& m = P.m;
    const DevOptics& o = P.o;

    // ---- Sec. 3.1: source -> point on the lens ----------------------------
    df Rx = sx, Ry = sy, Rz = sz;
    df dx, dy, dz;
    ray_start(P, sx, sy, sz, sid, rid, dx, dy, dz);
    int status = PIVBOS_RAY_REACHED;
    int steps = 0;
    out.w = 1.0f;
    if (st) st->opl = 0.0;
    if constexpr (EXT) {
        if (o.rad_mode) out.w = ray_radiance(o, dx.hi, dy.hi, dz.hi);
    }

    // ---- Sec. 3.2: through the density box ------------------------------
    if (m.present) {
        df tn;
        const bool enters = box_entry(m, Rx, Ry, Rz, dx, dy, dz, tn);
        if (enters) {
            const df R0x = df_fma(dx, tn, Rx);
            const df R0y = df_fma(dy, tn, Ry);
            const df R0z = df_fma(dz, tn, Rz);
            // reference line R0 + T0 t in grid units (double-float): g0 at
            // the entry, dG per full step
            const df ihx = dfk(m.inv_hd[0]), ihy = dfk(m.inv_hd[1]), ihz = dfk(m.inv_hd[2]);
            df grx = df_mul(df_sub(R0x, dfk(m.origin[0])), ihx);
            df gry = df_mul(df_sub(R0y, dfk(m.origin[1])), ihy);
            df grz = df_mul(df_sub(R0z, dfk(m.origin[2])), ihz);
            // n at the entry as double-float (1 + dn in FP32 would round the
            // tangent's length, hence the ray's parameter, by ~6e-8)
            const df n0 = df_add_f(dfv(1.0f), sample_field(m, grx.hi + grx.lo, gry.hi + gry.lo, grz.hi + grz.lo).x);
            // reading: no refraction at the faces; T = n d at the entry
            const df T0x = df_mul(dx, n0), T0y = df_mul(dy, n0), T0z = df_mul(dz, n0);
            const df dGx = df_mul(df_mul(T0x, ihx), dfk(P.step_df));
            const df dGy = df_mul(df_mul(T0y, ihy), dfk(P.step_df));
            const df dGz = df_mul(df_mul(T0z, ihz), dfk(P.step_df));
            const float T0fx = T0x.hi, T0fy = T0y.hi, T0fz = T0z.hi;
            const float ix = m.inv_h[0], iy = m.inv_h[1], iz = m.inv_h[2];
            float rhx = 0.f, rhy = 0.f, rhz = 0.f;   // position perturbation (m)
            float tax = 0.f, tay = 0.f, taz = 0.f;   // tangent perturbation
            const float hstep = P.step;
            const float ex = (float)(m.n[0] - 1), ey = (float)(m.n[1] - 1), ez = (float)(m.n[2] - 1);
            float h_last = 0.f;
            // optical path inside the box (exit states only): the integral of
            // n^2 dt = the parameter run plus the integral of n^2 - 1, the
            // latter by the stage weights (Simpson on the RK4 stage points,
            // the left rule for the first-order scheme), summed in double-float
            df opl_rest = dfv(0.f);
            int k = 0;
            bool done = false;
            CellCache<CACHE> cache;
            cache.reset();
            for (; k < P.max_steps; ++k) {
                // current point = reference (grx, gry, grz) + perturbation (cells)
                const float ox = fmaf(rhx, ix, grx.lo), oy = fmaf(rhy, iy, gry.lo), oz = fmaf(rhz, iz, grz.lo);
                const float Tx = T0fx + tax, Ty = T0fy + tay, Tz = T0fz + taz;
                // parameter distance to the box boundary along the tangent
                float dexit = INFINITY;
                if (Tx != 0.f) dexit = fminf(dexit, (Tx > 0.f ? (ex - grx.hi) - ox : -grx.hi - ox) * __fdividef(m.h[0], Tx));
                if (Ty != 0.f) dexit = fminf(dexit, (Ty > 0.f ? (ey - gry.hi) - oy : -gry.hi - oy) * __fdividef(m.h[1], Ty));
                if (Tz != 0.f) dexit = fminf(dexit, (Tz > 0.f ? (ez - grz.hi) - oz : -grz.hi - oz) * __fdividef(m.h[2], Tz));
                float h = hstep;
                if (hstep >= dexit) {
                    h = fmaxf(dexit, 0.f);
                    done = true;
                }
                // Stages of the step.  RK4 (Eqs. 3 and 5): K1 = A at the
                // start, K2 = B at (T/2 + A/8) h, K3 = C at (T + B/2) h;
                // rho += (tau + (A + 2B)/6) h, tau += (A + 4B + C)/6.
                // First-order scheme: one stage, rho += tau h, tau += A.
                float sRx = 0.f, sRy = 0.f, sRz = 0.f;   // sum of wR * K
                float sTx = 0.f, sTy = 0.f, sTz = 0.f;   // sum of wT * K
                float sQ = 0.f;                           // sum of wT * (n^2 - 1)
                float kx = 0.f, ky = 0.f, kz = 0.f;      // K of the previous stage
                constexpr int kStages = INTEG == PIVBOS_RK4 ? 3 : 1;
#pragma unroll
                for (int sg = 0; sg < kStages; ++sg) {
                    const float cT = sg == 0 ? 0.f : (sg == 1 ? 0.5f : 1.f);
                    const float cK = sg == 0 ? 0.f : (sg == 1 ? 0.125f : 0.5f);
                    const float px = (cT * Tx + cK * kx) * h;
                    const float py = (cT * Ty + cK * ky) * h;
                    const float pz = (cT * Tz + cK * kz) * h;
                    const float4 Dv = eval_D_split<CACHE>(m, cache, grx.hi, fmaf(px, ix, ox), gry.hi,
                                                          fmaf(py, iy, oy), grz.hi, fmaf(pz, iz, oz));
                    kx = Dv.x * h;
                    ky = Dv.y * h;
                    kz = Dv.z * h;
                    const float wR = INTEG == PIVBOS_RK4 ? (sg == 0 ? 1.f / 6.f : (sg == 1 ? 2.f / 6.f : 0.f)) : 0.f;
                    const float wT = INTEG == PIVBOS_RK4 ? (sg == 1 ? 4.f / 6.f : 1.f / 6.f) : 1.f;
                    sRx = fmaf(wR, kx, sRx); sRy = fmaf(wR, ky, sRy); sRz = fmaf(wR, kz, sRz);
                    sTx = fmaf(wT, kx, sTx); sTy = fmaf(wT, ky, sTy); sTz = fmaf(wT, kz, sTz);
                    if (st) sQ = fmaf(wT, Dv.w * (2.0f + Dv.w), sQ);   // n^2 - 1 = dn (2 + dn)
                }
                if (st) opl_rest = df_add_f(opl_rest, sQ * h);
                rhx = fmaf(tax + sRx, h, rhx);
                rhy = fmaf(tay + sRy, h, rhy);
                rhz = fmaf(taz + sRz, h, rhz);
                tax += sTx;
                tay += sTy;
                taz += sTz;
                if (done) {
                    h_last = h;
                    break;
                }
                grx = df_add(grx, dGx);
                gry = df_add(gry, dGy);
                grz = df_add(grz, dGz);
            }
            steps = done ? k + 1 : k;
            if (!done) status = PIVBOS_RAY_MAXSTEP;
            const df t_exit = df_add_f(df_mul_f(dfk(P.step_df), (float)k), h_last);
            if (st) st->opl = df_to_double(df_add(t_exit, opl_rest));
            Rx = df_add_f(df_add(R0x, df_mul(T0x, t_exit)), rhx);
            Ry = df_add_f(df_add(R0y, df_mul(T0y, t_exit)), rhy);
            Rz = df_add_f(df_add(R0z, df_mul(T0z, t_exit)), rhz);
            const df Tx = df_add_f(T0x, tax), Ty = df_add_f(T0y, tay), Tz = df_add_f(T0z, taz);
            const df inv = df_rsqrt(df_add(df_add(df_sqr(Tx), df_sqr(Ty)), df_sqr(Tz)));
            dx = df_mul(Tx, inv);
            dy = df_mul(Ty, inv);
            dz = df_mul(Tz, inv);
        }
    }
    if (st) {
        put3(st->vol_pos, Rx, Ry, Rz);
        put3(st->vol_dir, dx, dy, dz);
        st->steps = steps;
    }

    // ---- Sec. 3.3-3.4: optical elements and the sensor plane --------------
    df px, py;
    optics_to_sensor<DfOps, EXT>(o, Rx, Ry, Rz, dx, dy, dz, status, px, py);
    if (st) {
        st->sensor_xy[0] = df_to_double(px);
        st->sensor_xy[1] = df_to_double(py);
        put3(st->sensor_dir, dx, dy, dz);
        st->status = status;
    }
    out.px = px;
    out.py = py;
    out.status = status;
    out.steps = steps;
}

// ---------------------------------------------------------------------------
// Sec. 3.4 deposit weights: erf-integrated Gaussian over the pixels within
// 3 sigma (clipped to the sensor), renormalised over the window, quantised to
// 32.32 with the remainder on the largest weight (first in row-major order),
// so every ray adds exactly 2^32.
// ---------------------------------------------------------------------------
struct SpotWindow {
    int x0, y0, nx, ny;
    float wx[PIVBOS_MAX_WINDOW];
    float wy[PIVBOS_MAX_WINDOW];
    float scale;   // 2^32 / (sum wx * sum wy)
};

__device__ __forceinline__ void axis_weights(df p, float win3, int N, float inv_s2, int& lo, int& cnt, float* w,
                                             float& sum)
{
    float fa, fb;
    int a = df_floor(df_add_f(p, -win3), fa);
    int b = df_floor(df_add_f(p, win3), fb);
    a = max(a, 0);
    b = min(b, N - 1);
    lo = a;
    cnt = b - a + 1;
    // hit position relative to the window start (exact difference, then FP32)
    const float f = __fadd_rn(__fsub_rn(p.hi, (float)a), p.lo);
    float e_prev = erff((0.0f - f) * inv_s2);
    float fi = 1.0f;   // pixel edge index, exact in FP32
    sum = 0.f;
#pragma unroll 1
    for (int i = 0; i < cnt; ++i) {
        const float e_next = erff((fi - f) * inv_s2);
        w[i] = 0.5f * (e_next - e_prev);
        sum += w[i];
        e_prev = e_next;
        fi += 1.0f;
    }
}

__device__ __forceinline__ void spot_window(const DevOptics& o, df px, df py, SpotWindow& sw)
{
    float sx, sy;
    axis_weights(px, o.win3, o.W, o.inv_sqrt2_sigma, sw.x0, sw.nx, sw.wx, sx);
    axis_weights(py, o.win3, o.H, o.inv_sqrt2_sigma, sw.y0, sw.ny, sw.wy, sy);
    sw.scale = 4294967296.0f / (sx * sy);
}

constexpr int kTileW = 32;
constexpr int kTileH = 32;

__device__ __forceinline__ void add_q(unsigned long long* tile, int ax, int ay, int64_t* image, int W,
                                      int gx, int gy, unsigned long long q)
{
    const int tx = gx - ax, ty = gy - ay;
    if ((unsigned)tx < (unsigned)kTileW && (unsigned)ty < (unsigned)kTileH) {
        atomicAdd(&tile[ty * kTileW + tx], q);
    } else {
        atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * W + gx]), q);
    }
}

// The split tile: two planes of 32-bit cells, kTileW * kTileH each, holding
// for the values added to a pixel the sum of their low 16 bits and the sum
// of the rest (floor(v / 2^16), modulo 2^32: a remainder can be negative).
// The low sum is exact for up to 2^16 additions per pixel between flushes;
// the rest, read as a signed 32-bit number, is exact while the pixel's value
// stays below 2^47 (2^15 rays' worth), and the value is rest * 2^16 + low.  Many rays of a few sources
// land on the same pixels, and 32-bit shared-memory additions serialise on
// a shared address more cheaply than 64-bit ones.
__device__ __forceinline__ void add_q(uint32_t* tile, int ax, int ay, int64_t* image, int W, int gx, int gy,
                                      unsigned long long q)
{
    const int tx = gx - ax, ty = gy - ay;
    if ((unsigned)tx < (unsigned)kTileW && (unsigned)ty < (unsigned)kTileH) {
        const int c = ty * kTileW + tx;
        atomicAdd(&tile[c], (uint32_t)(q & 0xffffull));
        atomicAdd(&tile[kTileW * kTileH + c], (uint32_t)(q >> 16));
    } else {
        atomicAdd(reinterpret_cast<unsigned long long*>(&image[(size_t)gy * W + gx]), q);
    }
}

// Value of cell c of a split tile, and the cell cleared.
__device__ __forceinline__ unsigned long long take_split(uint32_t* tile, int c)
{
    const uint32_t lo = tile[c], hi = tile[kTileW * kTileH + c];
    if ((lo | hi) == 0u) return 0ull;
    tile[c] = 0u;
    tile[kTileW * kTileH + c] = 0u;
    return (unsigned long long)((long long)(int32_t)hi * 65536ll + (long long)lo);
}

// Round-to-nearest-even of a non-negative float below 2^33 to an integer
// with FP32/INT32 instructions only (the 64-bit float-to-integer conversion
// runs on GB300's narrow FP64 pipe).  Below 2^23 adding 2^23 rounds to an
// integer in the mantissa; from 2^23 up the float is already an integer.
__device__ __forceinline__ long long round_pos_to_ll(float x)
{
    if (x < 8388608.0f) return (long long)(__float_as_uint(x + 8388608.0f) - 0x4B000000u);
    const uint32_t b = __float_as_uint(x);
    return (long long)((b & 0x7FFFFFu) | 0x800000u) << ((int)(b >> 23) - 150);
}

// Warp-aggregated deposit (off by default): the lanes of `lanes` (all
// depositing, all executing this together) take their spots' pixels in
// step; lanes adding to the same pixel in a step are matched and one of
// them adds their sum, so a pixel that a warp's rays share costs one atomic
// instead of one per ray.  The 64-bit values (each below 2^33) are summed as
// 16-bit low and high parts, exact in 32 bits for up to 32 lanes.  Measured
// on GB300 it renders the same images bit for bit but 2.1x slower on the
// PIV workload (defocused particles: a warp's rays rarely share a pixel, so
// the match and reductions of every step buy nothing) and 3.1x slower in
// the surrogate's finish kernel; the plain per-lane shared-memory atomics
// stay.  Build with -DPIVBOS_DEPOSIT_AGG=1 to reproduce the measurement.
#ifndef PIVBOS_DEPOSIT_AGG
#define PIVBOS_DEPOSIT_AGG 0
#endif

// Quantise the spot of one ray and add it (tile if inside, image otherwise).
// WEIGHTED: the ray carries the radiance weight w in [0, 1] and adds
// round(w 2^32) in all; otherwise exactly 2^32.  lanes: the warp's lanes
// that deposit together (the caller's ballot), for the aggregated adds.
template <bool WEIGHTED = false, class TileT = unsigned long long>
__device__ __forceinline__ void deposit_ray(const DevOptics& o, df px, df py,
                                            TileT* tile, int ax, int ay, int64_t* image,
                                            float w = 1.0f, unsigned lanes = 0u)
{
    SpotWindow sw;
    spot_window(o, px, py, sw);
    long long total = 4294967296LL;
    if constexpr (WEIGHTED) {
        sw.scale *= w;
        total = round_pos_to_ll(w * 4294967296.0f);
    }
    long long sum = 0, qmax = -1;
    int imax = 0, jmax = 0;
#if !PIVBOS_DEPOSIT_AGG
    // One pass: every quantum is added as it is computed, then the rounding
    // remainder (of either sign) onto the first largest quantum's pixel --
    // the same pixel totals as adding it with that quantum (integer sums
    // commute; a negative remainder wraps in the 64-bit cells and, in the
    // split tile, in the 32-bit plane of the upper bits).
#pragma unroll 1
    for (int j = 0; j < sw.ny; ++j) {
        const float wyj = sw.wy[j] * sw.scale;
#pragma unroll 1
        for (int i = 0; i < sw.nx; ++i) {
            const long long q = round_pos_to_ll(sw.wx[i] * wyj);
            sum += q;
            if (q > qmax) { qmax = q; imax = i; jmax = j; }
            if (q != 0) add_q(tile, ax, ay, image, o.W, sw.x0 + i, sw.y0 + j, (unsigned long long)q);
        }
    }
    const long long rem = total - sum;
    if (rem != 0) add_q(tile, ax, ay, image, o.W, sw.x0 + imax, sw.y0 + jmax, (unsigned long long)rem);
#else
#pragma unroll 1
    for (int j = 0; j < sw.ny; ++j) {
        const float wyj = sw.wy[j] * sw.scale;
#pragma unroll 1
        for (int i = 0; i < sw.nx; ++i) {
            const long long q = round_pos_to_ll(sw.wx[i] * wyj);
            sum += q;
            if (q > qmax) { qmax = q; imax = i; jmax = j; }
        }
    }
    const long long rem = total - sum;
    if (lanes) {
        const int n = sw.nx * sw.ny;
        const int steps = (int)__reduce_max_sync(lanes, (unsigned)n);
        const uint32_t lane = threadIdx.x & 31;
        int i = 0, j = 0;
        float wyj = sw.wy[0] * sw.scale;
#pragma unroll 1
        for (int t = 0; t < steps; ++t) {
            uint32_t key = 0x80000000u | lane;   // no pixel: a group of its own
            unsigned long long q = 0ull;
            if (t < n) {
                long long v = round_pos_to_ll(sw.wx[i] * wyj);
                if (i == imax && j == jmax) v += rem;
                q = (unsigned long long)v;
                if (q) key = (uint32_t)(sw.y0 + j) * (uint32_t)o.W + (uint32_t)(sw.x0 + i);
            }
            const unsigned peers = __match_any_sync(lanes, key);
            const uint32_t lo = __reduce_add_sync(peers, (uint32_t)(q & 0xffffull));
            const uint32_t hi = __reduce_add_sync(peers, (uint32_t)(q >> 16));
            if (!(key & 0x80000000u) && lane == (uint32_t)(__ffs(peers) - 1))
                add_q(tile, ax, ay, image, o.W, sw.x0 + i, sw.y0 + j, ((unsigned long long)hi << 16) + lo);
            if (t < n && ++i == sw.nx) {
                i = 0;
                if (++j < sw.ny) wyj = sw.wy[j] * sw.scale;
            }
        }
        return;
    }
#pragma unroll 1
    for (int j = 0; j < sw.ny; ++j) {
        const float wyj = sw.wy[j] * sw.scale;
#pragma unroll 1
        for (int i = 0; i < sw.nx; ++i) {
            long long q = round_pos_to_ll(sw.wx[i] * wyj);
            if (i == imax && j == jmax) q += rem;
            if (q != 0) add_q(tile, ax, ay, image, o.W, sw.x0 + i, sw.y0 + j, (unsigned long long)q);
        }
    }
#endif
}


constexpr int kMaxOrderRays = 2048;   // a CTA reorders at most this many rays

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Ordering key of a ray: Morton code of the grid cell where its straight
// line from the source to its lens point crosses the mid-plane of the box
// (FP32 throughout -- only the order of tracing depends on it), above the
// ray's index within the CTA.
__device__ __forceinline__ uint32_t ray_order_key(const TraceParams& P, uint32_t flat, uint32_t local)
{
    const uint32_t rps = P.rays_per_source;
    const uint32_t slot = flat / rps, k = flat - slot * rps;
    const uint32_t sid = __ldg(P.perm + slot) + P.source_offset;
    const float2* sp = P.src_df + 3 * (size_t)slot;
    const float sx = __ldg(sp).x, sy = __ldg(sp + 1).x, sz = __ldg(sp + 2).x;
    uint64_t w0, w1;
    philox_lens_words(k, sid, P.frame, 0ull, P.seed, 0ull, w0, w1);
    const float u1 = ((float)(uint32_t)(w0 >> 40) + 0.5f) * 0x1p-24f;
    const float u2 = ((float)(uint32_t)(w1 >> 40) + 0.5f) * 0x1p-24f;
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    const float r = P.o.aim_r.hi * sqrtf(u1);
    const float dz = P.o.aim_z.hi - sz;
    const float t = dz != 0.0f ? fminf(fmaxf((P.m.z_key - sz) / dz, 0.0f), 1.0f) : 0.0f;
    const float x = fmaf(r * cs - sx, t, sx), y = fmaf(r * sn - sy, t, sy);
    const float gx = fminf(fmaxf((x - P.m.origin[0].hi) * P.m.inv_h[0], 0.0f), 1023.0f);
    const float gy = fminf(fmaxf((y - P.m.origin[1].hi) * P.m.inv_h[1], 0.0f), 1023.0f);
    const uint32_t code = spread10((uint32_t)gx) | (spread10((uint32_t)gy) << 1);
    return (code << 11) | local;
}

// Sort the n (<= kMaxOrderRays) rays of a chunk starting at list position
// `first` by ray_order_key; order[e] & 0x7ff is then the position of the
// e-th ray to trace.  Every thread of the CTA must call it.
__device__ __forceinline__ void order_chunk(const TraceParams& P, uint32_t* order, uint64_t first, uint32_t n)
{
    uint32_t n_pow2 = 1;
    while (n_pow2 < n) n_pow2 <<= 1;
    for (uint32_t q = threadIdx.x; q < n_pow2; q += blockDim.x)
        order[q] = q < n ? ray_order_key(P, P.ray_list ? __ldg(P.ray_list + first + q) : (uint32_t)(first + q), q)
                         : 0xffffffffu;
    __syncthreads();
    for (uint32_t kk = 2; kk <= n_pow2; kk <<= 1) {
        for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < n_pow2 / 2; t += blockDim.x) {
                const uint32_t i = 2 * t - (t & (j - 1));
                const uint32_t l = i + j;
                const bool up = (i & kk) == 0;
                const uint32_t a = order[i], b = order[l];
                if ((a > b) == up) {
                    order[i] = b;
                    order[l] = a;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace pivbos
