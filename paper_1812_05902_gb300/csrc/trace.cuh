// Device functions of the ray tracer: one GPU thread follows one ray through
// all four steps of the method (arXiv 1812.05902, Sec. 3 and Sec. 3.5).
//
// Precision plan (GB300 runs FP64 at a small fraction of FP32):
//  * lens point: FP64 from 53-bit uniforms (as the method draws it);
//  * straight runs, lens surfaces, sensor plane: FP64;
//  * integration: the ray is carried as a straight reference line
//    R0 + T0 t (FP64) plus an FP32 perturbation (rho, tau) that the
//    Runge-Kutta update acts on.  The update of Eq. 3 is linear in (R, T), so
//    R_i = R0 + T0 t_i + rho_i, T_i = T0 + tau_i gives exactly
//        rho_{i+1} = rho_i + [tau_i + (A + 2B)/6] dt,
//        tau_{i+1} = tau_i + (A + 4B + C)/6,
//    and the FP32 rounding applies to deflections (~1e-5 rad, ~1e-5 m) rather
//    than to absolute positions (~1 m) and directions (~1).
//  * sample positions for the field are FP32 grid coordinates (error
//    ~1e-5 of a cell), which only perturbs where n is evaluated.
#pragma once

#include <math.h>

#include "common.cuh"

namespace pivbos {

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

struct RayOut {
    double px, py;     // sensor pixel coordinates
    int status;
    int steps;
};

// ---------------------------------------------------------------------------
// One ray through all stages.  INTEG: PIVBOS_EULER or PIVBOS_RK4.  If st is
// not null the full exit state is written (parity path).
// ---------------------------------------------------------------------------
template <int INTEG>
__device__ __forceinline__ void trace_ray(const TraceParams& P, double sx, double sy, double sz,
                                          uint32_t sid, uint32_t rid, RayOut& out,
                                          pivbos_ray_state* st)
{
    const DevMedium& m = P.m;
    const DevOptics& o = P.o;

    // ---- Sec. 3.1: source -> point on the lens ----------------------------
    // 53-bit uniforms in (0,1); r = a sqrt(u1), phi = 2 pi u2 (FP64)
    uint64_t w0, w1;
    philox_lens_words(rid, sid, P.frame, 0ull, P.seed, 0ull, w0, w1);
    const double u1 = ((double)(w0 >> 11) + 0.5) * 0x1p-53;
    const double u2 = ((double)(w1 >> 11) + 0.5) * 0x1p-53;
    double sq_u1;
    {
        double y = (double)rsqrtf((float)u1);
        y = y * (1.5 - 0.5 * u1 * y * y);
        y = y * (1.5 - 0.5 * u1 * y * y);
        sq_u1 = u1 * y;
    }
    const double rr = o.aim_r * sq_u1;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    double Rx = sx, Ry = sy, Rz = sz;
    double dx = rr * cs - sx;
    double dy = rr * sn - sy;
    double dz = o.aim_z - sz;
    {
        const double l2 = dx * dx + dy * dy + dz * dz;
        double y = (double)rsqrtf((float)l2);
        y = y * (1.5 - 0.5 * l2 * y * y);   // two Newton steps in FP64
        y = y * (1.5 - 0.5 * l2 * y * y);
        dx *= y; dy *= y; dz *= y;
    }
    int status = PIVBOS_RAY_REACHED;
    int steps = 0;

    // ---- Sec. 3.2: through the density box ------------------------------
    if (m.present) {
        const bool inside = Rx >= m.lo[0] && Rx <= m.hi[0] && Ry >= m.lo[1] && Ry <= m.hi[1] &&
                            Rz >= m.lo[2] && Rz <= m.hi[2];
        bool enters = inside;
        double tn = 0.0;
        if (!inside) {
            // slab test on the straight line (FP64; the entry parameter only
            // moves the start point along the line)
            double t_near = -INFINITY, t_far = INFINITY;
            bool ok = true;
            const double dd[3] = {dx, dy, dz};
            const double RR[3] = {Rx, Ry, Rz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (dd[a] == 0.0) {
                    if (RR[a] < m.lo[a] || RR[a] > m.hi[a]) ok = false;
                } else {
                    const double inv = 1.0 / dd[a];
                    const double t1 = (m.lo[a] - RR[a]) * inv;
                    const double t2 = (m.hi[a] - RR[a]) * inv;
                    t_near = fmax(t_near, fmin(t1, t2));
                    t_far = fmin(t_far, fmax(t1, t2));
                }
            }
            if (ok && t_near <= t_far && t_near >= 0.0) {
                enters = true;
                tn = t_near;
            }
        }
        if (enters) {
            const double R0x = Rx + tn * dx, R0y = Ry + tn * dy, R0z = Rz + tn * dz;
            // grid coordinates of the entry point and of the reference line
            const float g0x = (float)((R0x - m.origin[0]) * m.inv_hd[0]);
            const float g0y = (float)((R0y - m.origin[1]) * m.inv_hd[1]);
            const float g0z = (float)((R0z - m.origin[2]) * m.inv_hd[2]);
            const float n0 = 1.0f + sample_field(m, g0x, g0y, g0z).x;
            // reading: no refraction at the faces; T = n d at the entry
            const double T0x = (double)n0 * dx, T0y = (double)n0 * dy, T0z = (double)n0 * dz;
            const float T0fx = (float)T0x, T0fy = (float)T0y, T0fz = (float)T0z;
            const float G0x = T0fx * m.inv_h[0], G0y = T0fy * m.inv_h[1], G0z = T0fz * m.inv_h[2];
            float rhx = 0.f, rhy = 0.f, rhz = 0.f;   // position perturbation (m)
            float tax = 0.f, tay = 0.f, taz = 0.f;   // tangent perturbation
            const float hstep = P.step;
            const float ex = (float)(m.n[0] - 1), ey = (float)(m.n[1] - 1), ez = (float)(m.n[2] - 1);
            float h_last = 0.f;
            int k = 0;
            bool done = false;
            for (; k < P.max_steps; ++k) {
                const float t = (float)k * hstep;
                const float gx = fmaf(G0x, t, g0x) + rhx * m.inv_h[0];
                const float gy = fmaf(G0y, t, g0y) + rhy * m.inv_h[1];
                const float gz = fmaf(G0z, t, g0z) + rhz * m.inv_h[2];
                const float Tx = T0fx + tax, Ty = T0fy + tay, Tz = T0fz + taz;
                // parameter distance to the box boundary along the tangent
                float dexit = INFINITY;
                if (Tx > 0.f) dexit = fminf(dexit, (ex - gx) * m.h[0] / Tx);
                else if (Tx < 0.f) dexit = fminf(dexit, -gx * m.h[0] / Tx);
                if (Ty > 0.f) dexit = fminf(dexit, (ey - gy) * m.h[1] / Ty);
                else if (Ty < 0.f) dexit = fminf(dexit, -gy * m.h[1] / Ty);
                if (Tz > 0.f) dexit = fminf(dexit, (ez - gz) * m.h[2] / Tz);
                else if (Tz < 0.f) dexit = fminf(dexit, -gz * m.h[2] / Tz);
                float h = hstep;
                if (hstep >= dexit) {
                    h = fmaxf(dexit, 0.f);
                    done = true;
                }
                if (INTEG == PIVBOS_RK4) {
                    // Eqs. 3 and 5
                    const float3 Dv = eval_D(m, gx, gy, gz);
                    const float Ax = Dv.x * h, Ay = Dv.y * h, Az = Dv.z * h;
                    const float bxp = (0.5f * Tx + 0.125f * Ax) * h;
                    const float byp = (0.5f * Ty + 0.125f * Ay) * h;
                    const float bzp = (0.5f * Tz + 0.125f * Az) * h;
                    const float3 Db = eval_D(m, fmaf(bxp, m.inv_h[0], gx), fmaf(byp, m.inv_h[1], gy),
                                             fmaf(bzp, m.inv_h[2], gz));
                    const float Bx = Db.x * h, By = Db.y * h, Bz = Db.z * h;
                    const float cxp = (Tx + 0.5f * Bx) * h;
                    const float cyp = (Ty + 0.5f * By) * h;
                    const float czp = (Tz + 0.5f * Bz) * h;
                    const float3 Dc = eval_D(m, fmaf(cxp, m.inv_h[0], gx), fmaf(cyp, m.inv_h[1], gy),
                                             fmaf(czp, m.inv_h[2], gz));
                    const float Cx = Dc.x * h, Cy = Dc.y * h, Cz = Dc.z * h;
                    const float s6 = 1.0f / 6.0f;
                    rhx = fmaf(tax + (Ax + 2.f * Bx) * s6, h, rhx);
                    rhy = fmaf(tay + (Ay + 2.f * By) * s6, h, rhy);
                    rhz = fmaf(taz + (Az + 2.f * Bz) * s6, h, rhz);
                    tax += (Ax + 4.f * Bx + Cx) * s6;
                    tay += (Ay + 4.f * By + Cy) * s6;
                    taz += (Az + 4.f * Bz + Cz) * s6;
                } else {
                    // first-order scheme: both updates from the old state
                    const float3 Dv = eval_D(m, gx, gy, gz);
                    rhx = fmaf(tax, h, rhx);
                    rhy = fmaf(tay, h, rhy);
                    rhz = fmaf(taz, h, rhz);
                    tax = fmaf(Dv.x, h, tax);
                    tay = fmaf(Dv.y, h, tay);
                    taz = fmaf(Dv.z, h, taz);
                }
                if (done) {
                    h_last = h;
                    break;
                }
            }
            steps = done ? k + 1 : k;
            if (!done) status = PIVBOS_RAY_MAXSTEP;
            const double t_exit = (double)k * P.step_d + (double)h_last;
            Rx = R0x + T0x * t_exit + (double)rhx;
            Ry = R0y + T0y * t_exit + (double)rhy;
            Rz = R0z + T0z * t_exit + (double)rhz;
            const double Tx = T0x + (double)tax, Ty = T0y + (double)tay, Tz = T0z + (double)taz;
            const double l2 = Tx * Tx + Ty * Ty + Tz * Tz;
            double y = (double)rsqrtf((float)l2);
            y = y * (1.5 - 0.5 * l2 * y * y);
            y = y * (1.5 - 0.5 * l2 * y * y);
            dx = Tx * y; dy = Ty * y; dz = Tz * y;
        }
    }
    if (st) {
        st->vol_pos[0] = Rx; st->vol_pos[1] = Ry; st->vol_pos[2] = Rz;
        st->vol_dir[0] = dx; st->vol_dir[1] = dy; st->vol_dir[2] = dz;
        st->steps = steps;
    }

    // ---- Sec. 3.3: optical elements in sequence (FP64) --------------------
    double n_cur = o.n_object;
    for (int s = 0; s < o.ns && status == PIVBOS_RAY_REACHED; ++s) {
        const DevSurface S = o.s[s];
        if (!(dz > 0.0)) { status = PIVBOS_RAY_MISS; break; }
        const double t0 = (S.z - Rz) / dz;
        if (S.type == PIVBOS_SURF_SPHERE && S.R != 0.0) {
            // vertex-relative quadratic t^2 + 2 b t + c = 0 from the point Q
            // on the vertex plane; the vertex-side root has the smaller
            // magnitude: t = c / (-b - sign(b) sqrt(b^2 - c))
            const double Qx = Rx + t0 * dx, Qy = Ry + t0 * dy;
            const double b = dx * Qx + dy * Qy - S.R * dz;
            const double c = Qx * Qx + Qy * Qy;
            const double disc = b * b - c;
            if (disc < 0.0) { status = PIVBOS_RAY_MISS; break; }
            const double sq = sqrt(disc);
            const double den = -b - (b >= 0.0 ? sq : -sq);
            const double t1 = den != 0.0 ? c / den : 0.0;
            if (t0 + t1 < 0.0) { status = PIVBOS_RAY_MISS; break; }
            const double Hx = Qx + t1 * dx, Hy = Qy + t1 * dy, Hz = t1 * dz;
            if (!((Hz - S.R) * S.R < 0.0)) { status = PIVBOS_RAY_MISS; break; }
            if (Hx * Hx + Hy * Hy > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
            const double invR = 1.0 / S.R;
            double Nx = Hx * invR, Ny = Hy * invR, Nz = (Hz - S.R) * invR;
            if (Nx * dx + Ny * dy + Nz * dz > 0.0) { Nx = -Nx; Ny = -Ny; Nz = -Nz; }
            // Eq. 7, vector form
            const double eta = n_cur / S.n_after;
            const double ci = -(Nx * dx + Ny * dy + Nz * dz);
            const double kk = 1.0 - eta * eta * (1.0 - ci * ci);
            if (kk < 0.0) { status = PIVBOS_RAY_TIR; break; }
            const double a = eta * ci - sqrt(kk);
            dx = eta * dx + a * Nx;
            dy = eta * dy + a * Ny;
            dz = eta * dz + a * Nz;
            Rx = Hx; Ry = Hy; Rz = S.z + Hz;
            n_cur = S.n_after;
        } else {
            if (t0 < 0.0) { status = PIVBOS_RAY_MISS; break; }
            Rx += t0 * dx; Ry += t0 * dy; Rz = S.z;
            const double r2 = Rx * Rx + Ry * Ry;
            if (S.type == PIVBOS_SURF_STOP) {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_STOP; break; }
            } else if (S.type == PIVBOS_SURF_IDEAL_THIN) {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
                const double invdz = 1.0 / dz;
                const double ux = dx * invdz - Rx / S.f;
                const double uy = dy * invdz - Ry / S.f;
                const double inn = 1.0 / sqrt(ux * ux + uy * uy + 1.0);
                dx = ux * inn; dy = uy * inn; dz = inn;
            } else {
                if (r2 > S.clear_r2) { status = PIVBOS_RAY_MISS; break; }
                // flat surface, normal (0, 0, -1)
                const double eta = n_cur / S.n_after;
                const double ci = dz;
                const double kk = 1.0 - eta * eta * (1.0 - ci * ci);
                if (kk < 0.0) { status = PIVBOS_RAY_TIR; break; }
                const double a = eta * ci - sqrt(kk);
                dx = eta * dx;
                dy = eta * dy;
                dz = eta * dz - a;
                n_cur = S.n_after;
            }
        }
    }

    // ---- Sec. 3.4: sensor plane -------------------------------------------
    double px = 0.0, py = 0.0;
    if (status == PIVBOS_RAY_REACHED) {
        if (!(dz > 0.0)) {
            status = PIVBOS_RAY_MISS;
        } else {
            const double t = (o.sensor_z - Rz) / dz;
            if (t < 0.0) {
                status = PIVBOS_RAY_MISS;
            } else {
                px = (Rx + t * dx) * o.inv_pitch + o.half_w;
                py = (Ry + t * dy) * o.inv_pitch + o.half_h;
                if (!(px >= 0.0 && px < (double)o.W && py >= 0.0 && py < (double)o.H))
                    status = PIVBOS_RAY_OFF_SENSOR;
            }
        }
    }
    if (st) {
        st->sensor_xy[0] = px; st->sensor_xy[1] = py;
        st->sensor_dir[0] = dx; st->sensor_dir[1] = dy; st->sensor_dir[2] = dz;
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

__device__ __forceinline__ void axis_weights(double p, double win3, int N, float inv_s2, int& lo,
                                             int& cnt, float* w, float& sum)
{
    int a = (int)floor(p - win3);
    int b = (int)floor(p + win3);
    a = max(a, 0);
    b = min(b, N - 1);
    lo = a;
    cnt = b - a + 1;
    const float f = (float)(p - (double)a);   // hit position inside the window
    float e_prev = erff((0.0f - f) * inv_s2);
    sum = 0.f;
#pragma unroll
    for (int i = 0; i < PIVBOS_MAX_WINDOW; ++i) {
        if (i < cnt) {
            const float e_next = erff(((float)(i + 1) - f) * inv_s2);
            w[i] = 0.5f * (e_next - e_prev);
            sum += w[i];
            e_prev = e_next;
        } else {
            w[i] = 0.f;
        }
    }
}

__device__ __forceinline__ void spot_window(const DevOptics& o, double px, double py, SpotWindow& sw)
{
    float sx, sy;
    axis_weights(px, o.win3, o.W, o.inv_sqrt2_sigma, sw.x0, sw.nx, sw.wx, sx);
    axis_weights(py, o.win3, o.H, o.inv_sqrt2_sigma, sw.y0, sw.ny, sw.wy, sy);
    sw.scale = 4294967296.0f / (sx * sy);
}

}  // namespace pivbos
