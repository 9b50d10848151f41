/*
 * pivbos oracle -- TEST INFRASTRUCTURE, not the product.
 *
 * A plain, slow, serial-per-ray FP64 restatement of the image generator of
 * Rajendran, Bane & Vlachos, "PIV/BOS Synthetic Image Generation in Variable
 * Density Environments" (arXiv 1812.05902).  It exists only so that the CUDA
 * library can be checked against something written independently from the
 * paper.  Only tests/, __graft_entry__.smoke() and the cpu_baseline leg of
 * bench.py may load it.  It shares no source with the CUDA path (its own
 * Philox, its own field preparation, its own optics).
 *
 * Stage map (paper Section 3, Fig. 2):
 *   om_philox4x64 / om_lens_point ....... Sec. 3.1 (light field generation)
 *   om_medium_build / om_sample ......... Sec. 3.2, Eq. 1 (Gladstone-Dale),
 *                                         Eq. 6 (gradient of n on the grid)
 *   om_trace (integration part) ......... Sec. 3.2, Eqs. 2-6 (Sharma RK4) and
 *                                         the first-order scheme of Sec. 3.2
 *   om_trace (optics part) .............. Sec. 3.3, Eq. 7 (Snell), apertures
 *   om_trace (sensor) / om_deposit ...... Sec. 3.4, Eq. 8 (diffraction spot)
 *   om_line_gradient_integral ........... Sec. 4, Eq. 9 (BOS theory deflection)
 *   om_mie / om_ray_weight .............. Sec. 3.1 (Mie radiance of a ray)
 *   om_advect / om_image_u16 ............ image pairs and 16-bit images
 *                                         (Sec. 3.4's dynamic range)
 *
 * Readings where the paper is silent (box faces, final step, windows,
 * quantisation, ideal lens) are documented at each function.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, library routines or brute force, except where a
 * comment says "parity unpinned".
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC
 * (-ffp-contract=off so that x86 and Arm give the same FP64 results.)
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OM_MAX_SURF 16

/* ray status codes (same numbering as the public header, written out here
 * independently) */
enum {
    OM_REACHED = 0,
    OM_KILLED_STOP = 1,      /* blocked by an aperture (Sec. 3.3, item 3) */
    OM_KILLED_MISS = 2,      /* missed a surface or its clear aperture */
    OM_KILLED_TIR = 3,       /* total internal reflection (Sec. 3.3, item 2) */
    OM_KILLED_OFF_SENSOR = 4,/* hit the sensor plane outside the pixel array */
    OM_KILLED_MAXSTEP = 5    /* integration step budget exhausted */
};

enum { OM_SURF_SPHERE = 0, OM_SURF_PLANE = 1, OM_SURF_IDEAL_THIN = 2, OM_SURF_STOP = 3,
       OM_SURF_MIRROR = 4, OM_SURF_LENS_ARRAY = 5 };
enum { OM_EULER = 0, OM_RK4 = 1 };

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Sec. 3.1 draws one lens point per ray; the    */
/* counter-based generator makes every ray's draw independent of order.    */
/* ------------------------------------------------------------------------ */
static void om_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void om_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    /* multipliers and Weyl key increments of Philox4x64 from the SC'11 paper */
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        om_mulhilo64(M0, c0, &hi0, &lo0);
        om_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64-bit word -> double uniform in the open interval (0,1): top 53 bits plus
 * one half, times 2^-53. */
double om_u01(uint64_t w)
{
    return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Sec. 3.1: a ray is the vector from its source to a point on the lens.
 * The lens point is drawn uniformly over the aiming disk (radius a, centred on
 * the optical axis at z = aim_z): r = a sqrt(u1), phi = 2 pi u2.  Counter =
 * (ray, source, frame, purpose 0); key = (seed, 0). */
void om_lens_point(uint64_t seed, uint32_t source_id, uint32_t ray_id, uint32_t frame,
                   double aim_r, double aim_z, double p[3])
{
    uint64_t ctr[4] = { ray_id, source_id, frame, 0 };
    uint64_t key[2] = { seed, 0 };
    uint64_t w[4];
    om_philox4x64(ctr, key, w);
    double u1 = om_u01(w[0]);
    double u2 = om_u01(w[1]);
    double r = aim_r * sqrt(u1);
    double phi = 2.0 * M_PI * u2;
    p[0] = r * cos(phi);
    p[1] = r * sin(phi);
    p[2] = aim_z;
}

/* ------------------------------------------------------------------------ */
/* Medium: Eq. 1 (n = K rho + 1) at grid nodes, gradient of n at the nodes   */
/* by second-order finite differences (the grid gradient Eq. 6 needs).      */
/* Nodes sit at origin + i * spacing, x fastest: index (k*ny + j)*nx + i.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n[3];
    double origin[3], spacing[3];
    double K;
    double *dn;     /* n - 1 = K rho at nodes */
    double *g[3];   /* dn/dx, dn/dy, dn/dz at nodes */
} om_medium;

static size_t om_idx(const om_medium *m, int i, int j, int k)
{
    return ((size_t)k * (size_t)m->n[1] + (size_t)j) * (size_t)m->n[0] + (size_t)i;
}

/* derivative of the node values f along one axis at node position q (0..N-1),
 * reading neighbours through get(q') -- central difference inside,
 * second-order one-sided at the two end nodes, two-point difference when the
 * axis has only two nodes. */
static double om_diff(const om_medium *m, int axis, int i, int j, int k)
{
    int N = m->n[axis];
    int q = axis == 0 ? i : (axis == 1 ? j : k);
    double h = m->spacing[axis];
#define OM_AT(qq) m->dn[axis == 0 ? om_idx(m, (qq), j, k) : (axis == 1 ? om_idx(m, i, (qq), k) : om_idx(m, i, j, (qq)))]
    double d;
    if (N == 2) {
        d = (OM_AT(1) - OM_AT(0)) / h;
    } else if (q == 0) {
        d = (-3.0 * OM_AT(0) + 4.0 * OM_AT(1) - OM_AT(2)) / (2.0 * h);
    } else if (q == N - 1) {
        d = (3.0 * OM_AT(N - 1) - 4.0 * OM_AT(N - 2) + OM_AT(N - 3)) / (2.0 * h);
    } else {
        d = (OM_AT(q + 1) - OM_AT(q - 1)) / (2.0 * h);
    }
#undef OM_AT
    return d;
}

om_medium *om_medium_build(const float *rho, int nx, int ny, int nz,
                           const double origin[3], const double spacing[3], double K)
{
    if (nx < 2 || ny < 2 || nz < 2) return NULL;
    om_medium *m = (om_medium *)calloc(1, sizeof(om_medium));
    m->n[0] = nx; m->n[1] = ny; m->n[2] = nz;
    for (int a = 0; a < 3; ++a) { m->origin[a] = origin[a]; m->spacing[a] = spacing[a]; }
    m->K = K;
    size_t N = (size_t)nx * ny * nz;
    m->dn = (double *)malloc(N * sizeof(double));
    for (int a = 0; a < 3; ++a) m->g[a] = (double *)malloc(N * sizeof(double));
    /* Eq. 1 */
    for (size_t p = 0; p < N; ++p) m->dn[p] = K * (double)rho[p];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                for (int a = 0; a < 3; ++a)
                    m->g[a][om_idx(m, i, j, k)] = om_diff(m, a, i, j, k);
    return m;
}

void om_medium_free(om_medium *m)
{
    if (!m) return;
    free(m->dn);
    for (int a = 0; a < 3; ++a) free(m->g[a]);
    free(m);
}

/* copy out the node arrays (for tests) */
void om_medium_nodes(const om_medium *m, double *dn, double *gx, double *gy, double *gz)
{
    size_t N = (size_t)m->n[0] * m->n[1] * m->n[2];
    memcpy(dn, m->dn, N * sizeof(double));
    memcpy(gx, m->g[0], N * sizeof(double));
    memcpy(gy, m->g[1], N * sizeof(double));
    memcpy(gz, m->g[2], N * sizeof(double));
}

/* Trilinear interpolation of n-1 and of each gradient component at point x,
 * with the point clamped into the box.  Sec. 3.2 evaluates n and its
 * gradient at the ray position from the grid ("the grid point corresponding
 * to the given location of the ray"); trilinear sampling is how a position
 * between nodes is given a value. */
void om_sample(const om_medium *m, const double x[3], double *dn, double g[3])
{
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (x[a] - m->origin[a]) / m->spacing[a];
        if (u < 0.0) u = 0.0;
        if (u > (double)(m->n[a] - 1)) u = (double)(m->n[a] - 1);
        int i = (int)floor(u);
        if (i > m->n[a] - 2) i = m->n[a] - 2;
        i0[a] = i;
        f[a] = u - (double)i;
    }
    double acc_dn = 0.0, acc_g[3] = { 0.0, 0.0, 0.0 };
    for (int c = 0; c < 8; ++c) {
        int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        size_t p = om_idx(m, i0[0] + di, i0[1] + dj, i0[2] + dk);
        acc_dn += w * m->dn[p];
        for (int a = 0; a < 3; ++a) acc_g[a] += w * m->g[a][p];
    }
    *dn = acc_dn;
    for (int a = 0; a < 3; ++a) g[a] = acc_g[a];
}

/* Eq. 6: D = n grad(n), using the first form (n times the sampled gradient). */
static void om_D(const om_medium *m, const double R[3], double D[3])
{
    double dn, g[3];
    om_sample(m, R, &dn, g);
    double n = 1.0 + dn;
    for (int a = 0; a < 3; ++a) D[a] = n * g[a];
}

/* ------------------------------------------------------------------------ */
/* Optics (Sec. 3.3) and sensor (Sec. 3.4)                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int type;
    double z;        /* vertex (or plane) position on the axis */
    double R;        /* signed radius of curvature, centre at z + R (spheres,
                      * mirrors); the lenslet pitch of a lens array */
    double f;        /* focal length (ideal thin lens) */
    double n_after;  /* refractive index after the surface */
    double clear_r;  /* clear (or stop) radius */
} om_surface;

typedef struct {
    int ns;
    om_surface s[OM_MAX_SURF];
    double n_object;        /* index of the space the rays start in */
    double aim_z, aim_r;    /* disk the lens points are drawn on (Sec. 3.1) */
    double sensor_z, pitch;
    int W, H;
    double sigma;           /* Gaussian sigma of the spot, metres (d_tau/4) */
    /* sensor orientation: pixel axes eu, ev and normal en, the unit vectors
     * x, y, z turned by tilt_x about x, then by tilt_y about y; the sensor
     * centre stays at (0, 0, sensor_z) */
    double eu[3], ev[3], en[3];
    /* Mie radiance (Sec. 3.1): 0 = none (every ray weighs 1), 1 = unpolarised
     * laser, 2 = linearly polarised along pol; table of |S1|^2, |S2|^2 at
     * n_rad angles from 0 to pi; laser along L */
    int rad_mode, n_rad;
    double *rad;
    double L[3], pol[3], rad_max;
} om_optics;

typedef struct {
    double vol_pos[3], vol_dir[3];
    double sensor_xy[2];
    double sensor_dir[3];
    int32_t status, steps;
    double opl;   /* optical path inside the box, integral of n ds (0 if the ray never enters it) */
} om_ray_state;

/* Eq. 8 as printed (rule 0: 2.44 pi f# (M+1) lambda) or the textbook Airy
 * diameter (rule 1: 2.44 f# (M+1) lambda).  The spot is a Gaussian whose
 * e^-2 diameter is d_tau, so sigma = d_tau / 4. */
double om_sigma_from_eq8(double f_number, double M, double lambda, int rule)
{
    double dtau = 2.44 * (rule == 0 ? M_PI : 1.0) * f_number * (M + 1.0) * lambda;
    return dtau / 4.0;
}

om_optics *om_optics_build(const double *surf /* [ns][6]: type z R f n_after clear_r */, int ns,
                           double n_object, double aim_z, double aim_r,
                           double sensor_z, double pitch, int W, int H, double sigma)
{
    if (ns < 0 || ns > OM_MAX_SURF) return NULL;
    om_optics *o = (om_optics *)calloc(1, sizeof(om_optics));
    o->ns = ns;
    for (int i = 0; i < ns; ++i) {
        o->s[i].type = (int)surf[6 * i + 0];
        o->s[i].z = surf[6 * i + 1];
        o->s[i].R = surf[6 * i + 2];
        o->s[i].f = surf[6 * i + 3];
        o->s[i].n_after = surf[6 * i + 4];
        o->s[i].clear_r = surf[6 * i + 5];
    }
    o->n_object = n_object;
    o->aim_z = aim_z; o->aim_r = aim_r;
    o->sensor_z = sensor_z; o->pitch = pitch; o->W = W; o->H = H;
    o->sigma = sigma;
    o->eu[0] = 1.0; o->ev[1] = 1.0; o->en[2] = 1.0;
    return o;
}

/* Fig. 1(d) (perspective) and the Scheimpflug arrangement need a sensor that
 * is not square to the axis: turn the sensor about its centre, first by
 * tilt_x (radians) about the x axis, then by tilt_y about the y axis. */
void om_optics_tilt_sensor(om_optics *o, double tilt_x, double tilt_y)
{
    double cx = cos(tilt_x), sx = sin(tilt_x), cy = cos(tilt_y), sy = sin(tilt_y);
    /* R = Ry(tilt_y) Rx(tilt_x); columns are the turned x, y, z axes */
    double Rm[3][3] = { { cy, sy * sx, sy * cx }, { 0.0, cx, -sx }, { -sy, cy * sx, cy * cx } };
    for (int a = 0; a < 3; ++a) {
        o->eu[a] = Rm[a][0];
        o->ev[a] = Rm[a][1];
        o->en[a] = Rm[a][2];
    }
}

void om_optics_free(om_optics *o)
{
    if (o) free(o->rad);
    free(o);
}

/* Eq. 7 in vector form.  N is the unit surface normal facing the incoming
 * ray (N.d < 0).  Returns 0 on total internal reflection (the ray is then
 * killed -- the paper only says TIR must be considered). */
int om_refract(const double d[3], const double N[3], double n_i, double n_f, double out[3])
{
    double eta = n_i / n_f;
    double ci = -(N[0] * d[0] + N[1] * d[1] + N[2] * d[2]);
    double k = 1.0 - eta * eta * (1.0 - ci * ci);
    if (k < 0.0) return 0;
    double a = eta * ci - sqrt(k);
    for (int q = 0; q < 3; ++q) out[q] = eta * d[q] + a * N[q];
    return 1;
}

/* Sec. 3.3, item 1: the law of reflection about the unit normal N,
 * d' = d - 2 (d.N) N. */
void om_reflect(const double d[3], const double N[3], double out[3])
{
    double dn = d[0] * N[0] + d[1] * N[1] + d[2] * N[2];
    for (int q = 0; q < 3; ++q) out[q] = d[q] - 2.0 * dn * N[q];
}

/* move the point P along d to the plane z = zp; 0 if the plane is behind */
static int om_to_plane(double P[3], const double d[3], double zp)
{
    if (!(d[2] > 0.0)) return 0;
    double t = (zp - P[2]) / d[2];
    if (t < 0.0) return 0;
    P[0] += t * d[0];
    P[1] += t * d[1];
    P[2] = zp;
    return 1;
}

/* Sec. 3.3: intersect with a spherical surface given by its vertex on the
 * axis and signed radius.  The ray is first moved to the vertex plane; with
 * Q the point there relative to the vertex (Q_z = 0) the hit parameter solves
 * t^2 + 2 b t + c = 0, b = d.Q - R d_z, c = |Q|^2, and the root on the
 * vertex-side cap is the one of smaller magnitude, c / (-b - sign(b) sqrt(b^2 - c)).
 * Returns 0 on a miss. */
int om_sphere_hit(double P[3], const double d[3], double zv, double R, double N[3])
{
    double t0;
    if (!(d[2] > 0.0)) return 0;
    t0 = (zv - P[2]) / d[2];
    double Q[3] = { P[0] + t0 * d[0], P[1] + t0 * d[1], 0.0 };
    double b = d[0] * Q[0] + d[1] * Q[1] - R * d[2];
    double c = Q[0] * Q[0] + Q[1] * Q[1];
    double disc = b * b - c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double denom = -b - (b >= 0.0 ? sq : -sq);
    double t1 = denom != 0.0 ? c / denom : 0.0;
    if (t0 + t1 < 0.0) return 0;
    double H[3] = { Q[0] + t1 * d[0], Q[1] + t1 * d[1], t1 * d[2] };
    /* must lie on the hemisphere that contains the vertex */
    if (!((H[2] - R) * R < 0.0)) return 0;
    /* unit normal (H - C)/R, C = (0,0,R); orient it against the ray */
    double Nn[3] = { H[0] / R, H[1] / R, (H[2] - R) / R };
    double s = Nn[0] * d[0] + Nn[1] * d[1] + Nn[2] * d[2];
    if (s > 0.0) { Nn[0] = -Nn[0]; Nn[1] = -Nn[1]; Nn[2] = -Nn[2]; }
    P[0] = H[0]; P[1] = H[1]; P[2] = zv + H[2];
    N[0] = Nn[0]; N[1] = Nn[1]; N[2] = Nn[2];
    return 1;
}

/* ------------------------------------------------------------------------ */
/* One ray, all four stages (Sec. 3, Fig. 2).                               */
/* ------------------------------------------------------------------------ */
int om_max_steps(const om_medium *m, double step)
{
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double L = (double)(m->n[a] - 1) * m->spacing[a];
        diag2 += L * L;
    }
    return (int)ceil(2.0 * sqrt(diag2) / step) + 4;
}

/* Sec. 3.3 and 3.4: from point R, direction d in object space through the
 * optical elements in sequence, then onto the sensor.  Mirrors are coaxial
 * and the system is unfolded at each one: after the reflection the ray and
 * everything downstream are described in the frame mirrored about the
 * mirror's vertex plane (z -> 2 z_vertex - z), so light keeps travelling
 * toward +z and later elements are placed at larger z. */
static int om_optics_to_sensor(const om_optics *o, double R[3], double d[3], int status, om_ray_state *out)
{
    double n_cur = o->n_object;
    for (int s = 0; s < o->ns && status == OM_REACHED; ++s) {
        const om_surface *S = &o->s[s];
        if ((S->type == OM_SURF_SPHERE || S->type == OM_SURF_MIRROR) && S->R != 0.0) {
            double N[3], dn2[3];
            if (!om_sphere_hit(R, d, S->z, S->R, N)) { status = OM_KILLED_MISS; break; }
            if (R[0] * R[0] + R[1] * R[1] > S->clear_r * S->clear_r) { status = OM_KILLED_MISS; break; }
            if (S->type == OM_SURF_MIRROR) {
                om_reflect(d, N, dn2);
                /* unfold about the vertex plane */
                R[2] = 2.0 * S->z - R[2];
                d[0] = dn2[0]; d[1] = dn2[1]; d[2] = -dn2[2];
                continue;
            }
            if (!om_refract(d, N, n_cur, S->n_after, dn2)) { status = OM_KILLED_TIR; break; }
            for (int a = 0; a < 3; ++a) d[a] = dn2[a];
            n_cur = S->n_after;
        } else {
            if (!om_to_plane(R, d, S->z)) { status = OM_KILLED_MISS; break; }
            double r2 = R[0] * R[0] + R[1] * R[1];
            if (S->type == OM_SURF_STOP) {
                if (r2 > S->clear_r * S->clear_r) { status = OM_KILLED_STOP; break; }
            } else if (S->type == OM_SURF_MIRROR) {
                /* flat mirror square to the axis: reflection and unfolding
                 * about its own plane leave the ray as it was */
                if (r2 > S->clear_r * S->clear_r) { status = OM_KILLED_MISS; break; }
            } else if (S->type == OM_SURF_IDEAL_THIN || S->type == OM_SURF_LENS_ARRAY) {
                /* reading: an ideal (perfectly stigmatic) thin lens acting on
                 * the slopes, u' = u - (x - c) / f, c its centre; a lens array
                 * (Sec. 3.3: "an array of lenses as in a Plenoptic camera") is
                 * a square grid of such lenslets of pitch p centred at
                 * (i p, j p), the ray using the lenslet whose cell holds it */
                if (r2 > S->clear_r * S->clear_r) { status = OM_KILLED_MISS; break; }
                double cx = 0.0, cy = 0.0;
                if (S->type == OM_SURF_LENS_ARRAY) {
                    cx = S->R * floor(R[0] / S->R + 0.5);
                    cy = S->R * floor(R[1] / S->R + 0.5);
                }
                double sx = d[0] / d[2] - (R[0] - cx) / S->f;
                double sy = d[1] / d[2] - (R[1] - cy) / S->f;
                double nn = sqrt(sx * sx + sy * sy + 1.0);
                d[0] = sx / nn; d[1] = sy / nn; d[2] = 1.0 / nn;
            } else { /* flat refracting surface (sphere with R = 0 too) */
                if (r2 > S->clear_r * S->clear_r) { status = OM_KILLED_MISS; break; }
                double N[3] = { 0.0, 0.0, -1.0 }, dn2[3];
                if (!om_refract(d, N, n_cur, S->n_after, dn2)) { status = OM_KILLED_TIR; break; }
                for (int a = 0; a < 3; ++a) d[a] = dn2[a];
                n_cur = S->n_after;
            }
        }
    }

    /* Sec. 3.4: line-plane intersection with the sensor (through
     * (0, 0, sensor_z), normal en); pixel (i, j) covers [i, i+1) x [j, j+1)
     * along the sensor axes eu, ev, with the sensor centre at the array
     * centre */
    double px = 0.0, py = 0.0;
    if (status == OM_REACHED) {
        double dn = d[0] * o->en[0] + d[1] * o->en[1] + d[2] * o->en[2];
        double C[3] = { -R[0], -R[1], o->sensor_z - R[2] };   /* sensor centre - R */
        double t = (C[0] * o->en[0] + C[1] * o->en[1] + C[2] * o->en[2]) / dn;
        if (!(dn > 0.0) || t < 0.0) status = OM_KILLED_MISS;
        else {
            for (int a = 0; a < 3; ++a) R[a] += t * d[a];
            double X[3] = { R[0], R[1], R[2] - o->sensor_z };  /* hit - sensor centre */
            px = (X[0] * o->eu[0] + X[1] * o->eu[1] + X[2] * o->eu[2]) / o->pitch + 0.5 * (double)o->W;
            py = (X[0] * o->ev[0] + X[1] * o->ev[1] + X[2] * o->ev[2]) / o->pitch + 0.5 * (double)o->H;
            if (!(px >= 0.0 && px < (double)o->W && py >= 0.0 && py < (double)o->H))
                status = OM_KILLED_OFF_SENSOR;
        }
    }
    if (out) {
        out->sensor_xy[0] = px; out->sensor_xy[1] = py;
        for (int a = 0; a < 3; ++a) out->sensor_dir[a] = d[a];
        out->status = status;
    }
    return status;
}

/* The optics and sensor stages alone, from a given point and unit direction
 * in object space (for tests). */
int om_trace_optics(const om_optics *o, const double P[3], const double d_in[3], om_ray_state *out)
{
    double R[3] = { P[0], P[1], P[2] }, d[3] = { d_in[0], d_in[1], d_in[2] };
    for (int a = 0; a < 3; ++a) { out->vol_pos[a] = P[a]; out->vol_dir[a] = d_in[a]; }
    out->steps = 0;
    out->opl = 0.0;
    return om_optics_to_sensor(o, R, d, OM_REACHED, out);
}

int om_trace(const om_medium *m, const om_optics *o, const double src[3],
             uint64_t seed, uint32_t source_id, uint32_t ray_id, uint32_t frame,
             int integrator, double step, om_ray_state *out)
{
    double R[3], d[3], p[3];
    int status = OM_REACHED, steps = 0;
    /* Reading of the task's "path-length accumulation across the volume": the
     * optical path inside the box, integral of n ds.  With Sharma's parameter
     * (dt = ds / n, so ds = n dt) it is the integral of n^2 dt, taken along
     * the integrated path: Simpson's rule on the Runge-Kutta stage points
     * (t, t + h/2, t + h) for Eqs. 3-5, the left rule for the first-order
     * scheme. */
    double opl = 0.0;

    /* Sec. 3.1: origin = source, direction = unit vector to the lens point */
    om_lens_point(seed, source_id, ray_id, frame, o->aim_r, o->aim_z, p);
    double L2 = 0.0;
    for (int a = 0; a < 3; ++a) { R[a] = src[a]; d[a] = p[a] - src[a]; L2 += d[a] * d[a]; }
    double L = sqrt(L2);
    for (int a = 0; a < 3; ++a) d[a] /= L;

    /* Sec. 3.2: straight outside the grid (no gradient there), Eqs. 3-6 inside.
     * Reading: no refraction at the box faces; T = n(R) d at the entry. */
    if (m) {
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = m->origin[a];
            hi[a] = m->origin[a] + (double)(m->n[a] - 1) * m->spacing[a];
        }
        int inside = 1;
        for (int a = 0; a < 3; ++a) if (R[a] < lo[a] || R[a] > hi[a]) inside = 0;
        int enters = inside;
        if (!inside) {
            double tn = -INFINITY, tf = INFINITY;
            int ok = 1;
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.0) {
                    if (R[a] < lo[a] || R[a] > hi[a]) ok = 0;
                } else {
                    double t1 = (lo[a] - R[a]) / d[a];
                    double t2 = (hi[a] - R[a]) / d[a];
                    double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
                    if (tmin > tn) tn = tmin;
                    if (tmax < tf) tf = tmax;
                }
            }
            if (ok && tn <= tf && tn >= 0.0) {
                enters = 1;
                for (int a = 0; a < 3; ++a) R[a] += tn * d[a];
            }
        }
        if (enters) {
            double dn, g[3];
            om_sample(m, R, &dn, g);
            double T[3];
            for (int a = 0; a < 3; ++a) T[a] = (1.0 + dn) * d[a];
            int maxs = om_max_steps(m, step);
            int done = 0;
            for (int k = 0; k < maxs && !done; ++k) {
                /* reading: before each step, the parameter distance to the box
                 * boundary along the current tangent; if a full step would reach
                 * it, take one shortened final step that ends on the face. */
                double dexit = INFINITY;
                for (int a = 0; a < 3; ++a) {
                    if (T[a] > 0.0) { double q = (hi[a] - R[a]) / T[a]; if (q < dexit) dexit = q; }
                    else if (T[a] < 0.0) { double q = (lo[a] - R[a]) / T[a]; if (q < dexit) dexit = q; }
                }
                double h = step;
                if (step >= dexit) { h = dexit > 0.0 ? dexit : 0.0; done = 1; }
                if (integrator == OM_RK4) {
                    /* Eqs. 3 and 5 (Sharma et al.'s Runge-Kutta-Nystrom step) */
                    double A[3], B[3], C[3], X[3], nA, nB, nC, gq[3];
                    om_D(m, R, A);
                    om_sample(m, R, &nA, gq);
                    for (int a = 0; a < 3; ++a) A[a] *= h;
                    for (int a = 0; a < 3; ++a) X[a] = R[a] + (0.5 * T[a] + A[a] / 8.0) * h;
                    om_D(m, X, B);
                    om_sample(m, X, &nB, gq);
                    for (int a = 0; a < 3; ++a) B[a] *= h;
                    for (int a = 0; a < 3; ++a) X[a] = R[a] + (T[a] + 0.5 * B[a]) * h;
                    om_D(m, X, C);
                    om_sample(m, X, &nC, gq);
                    for (int a = 0; a < 3; ++a) C[a] *= h;
                    nA += 1.0; nB += 1.0; nC += 1.0;
                    opl += h / 6.0 * (nA * nA + 4.0 * nB * nB + nC * nC);
                    for (int a = 0; a < 3; ++a) {
                        R[a] = R[a] + (T[a] + (A[a] + 2.0 * B[a]) / 6.0) * h;
                        T[a] = T[a] + (A[a] + 4.0 * B[a] + C[a]) / 6.0;
                    }
                } else {
                    /* first-order (piecewise-linear) scheme: both updates from
                     * the state at the start of the step */
                    double Dv[3], nA, gq[3];
                    om_D(m, R, Dv);
                    om_sample(m, R, &nA, gq);
                    nA += 1.0;
                    opl += h * nA * nA;
                    for (int a = 0; a < 3; ++a) {
                        R[a] = R[a] + T[a] * h;
                        T[a] = T[a] + Dv[a] * h;
                    }
                }
                ++steps;
            }
            if (!done) status = OM_KILLED_MAXSTEP;
            double Tn = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
            for (int a = 0; a < 3; ++a) d[a] = T[a] / Tn;
        }
    }
    if (out) {
        for (int a = 0; a < 3; ++a) { out->vol_pos[a] = R[a]; out->vol_dir[a] = d[a]; }
        out->steps = steps;
        out->opl = opl;
    }

    return om_optics_to_sensor(o, R, d, status, out);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: the radiance of a ray from a PIV particle follows Mie          */
/* scattering (the paper computes it with Bohren & Huffman's method).  The  */
/* series solution for a homogeneous sphere of size parameter x = pi d /   */
/* lambda (wavelength in the medium) and relative index m:                  */
/*   a_n, b_n from the Riccati-Bessel functions psi_n(x) = x j_n(x),        */
/*   xi_n(x) = x h_n(x) = psi_n - i chi_n (upward recurrences from n = -1,  */
/*   0) and the logarithmic derivative D_n(mx) = psi_n'(mx) / psi_n(mx)     */
/*   (downward recurrence, started well above the last order);             */
/*   S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),                       */
/*   S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n), with the angular      */
/*   functions pi_n, tau_n of mu = cos(theta) by their recurrences;         */
/*   Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n),                              */
/*   Q_sca = (2/x^2) sum (2n+1) (|a_n|^2 + |b_n|^2);                        */
/*   the series stops after x + 4 x^(1/3) + 2 terms.                        */
/* s12[2i], s12[2i+1] = |S1|^2, |S2|^2 at theta_i = pi i / (n_angles - 1);  */
/* q = {Q_ext, Q_sca, Re S(0), n_terms}.  Returns the number of terms, 0 on */
/* bad input.                                                               */
/* ------------------------------------------------------------------------ */
int om_mie(double x, double m_re, double m_im, int n_angles, double *s12, double *q)
{
    if (!(x > 0.0) || !(m_re > 0.0) || n_angles < 2) return 0;
    double complex m = m_re + I * m_im;
    int nstop = (int)(x + 4.0 * cbrt(x) + 2.0);
    double mx = cabs(m * x);
    int nmx = (int)fmax((double)nstop, mx) + 16;
    double complex *D = (double complex *)calloc((size_t)nmx + 1, sizeof(double complex));
    double complex *a = (double complex *)calloc((size_t)nstop + 1, sizeof(double complex));
    double complex *b = (double complex *)calloc((size_t)nstop + 1, sizeof(double complex));
    double complex z = m * x;
    D[nmx] = 0.0;
    for (int n = nmx; n >= 1; --n) D[n - 1] = (double)n / z - 1.0 / (D[n] + (double)n / z);
    double psi_m1 = cos(x), psi_0 = sin(x);      /* psi_{-1}, psi_0 */
    double chi_m1 = -sin(x), chi_0 = cos(x);     /* chi_{-1}, chi_0 */
    double qe = 0.0, qs = 0.0;
    for (int n = 1; n <= nstop; ++n) {
        double psi_n = (2.0 * n - 1.0) / x * psi_0 - psi_m1;
        double chi_n = (2.0 * n - 1.0) / x * chi_0 - chi_m1;
        double complex xi_n = psi_n - I * chi_n, xi_p = psi_0 - I * chi_0;
        double complex ta = D[n] / m + (double)n / x;
        double complex tb = m * D[n] + (double)n / x;
        a[n] = (ta * psi_n - psi_0) / (ta * xi_n - xi_p);
        b[n] = (tb * psi_n - psi_0) / (tb * xi_n - xi_p);
        qe += (2.0 * n + 1.0) * creal(a[n] + b[n]);
        qs += (2.0 * n + 1.0) * (creal(a[n]) * creal(a[n]) + cimag(a[n]) * cimag(a[n]) +
                                 creal(b[n]) * creal(b[n]) + cimag(b[n]) * cimag(b[n]));
        psi_m1 = psi_0; psi_0 = psi_n;
        chi_m1 = chi_0; chi_0 = chi_n;
    }
    double complex s_fwd = 0.0;
    for (int i = 0; i < n_angles; ++i) {
        double th = M_PI * (double)i / (double)(n_angles - 1);
        double mu = cos(th);
        double pi_prev = 0.0, pi_n = 1.0;   /* pi_0, pi_1 */
        double complex S1 = 0.0, S2 = 0.0;
        for (int n = 1; n <= nstop; ++n) {
            double tau_n = n * mu * pi_n - (n + 1.0) * pi_prev;
            double f = (2.0 * n + 1.0) / ((double)n * (n + 1.0));
            S1 += f * (a[n] * pi_n + b[n] * tau_n);
            S2 += f * (a[n] * tau_n + b[n] * pi_n);
            double pi_next = ((2.0 * n + 1.0) / n) * mu * pi_n - ((n + 1.0) / n) * pi_prev;
            pi_prev = pi_n;
            pi_n = pi_next;
        }
        if (i == 0) s_fwd = S1;
        s12[2 * i] = creal(S1) * creal(S1) + cimag(S1) * cimag(S1);
        s12[2 * i + 1] = creal(S2) * creal(S2) + cimag(S2) * cimag(S2);
    }
    if (q) {
        q[0] = 2.0 / (x * x) * qe;
        q[1] = 2.0 / (x * x) * qs;
        q[2] = creal(s_fwd);
        q[3] = nstop;
    }
    free(D); free(a); free(b);
    return nstop;
}

/* Give the optics a Mie radiance: the table of |S1|^2, |S2|^2 over n
 * angles (om_mie), the laser direction L (unit) and, for a linearly
 * polarised laser, its polarisation pol (unit, normal to L; NULL =
 * unpolarised).  A ray leaving its source along d0 scatters by theta =
 * acos(d0.L); |S1|^2 and |S2|^2 are interpolated linearly in theta; its
 * radiance is |S2|^2 cos^2(phi) + |S1|^2 sin^2(phi) (phi between pol and
 * the scattering plane; unpolarised: the mean of the two) divided by the
 * largest entry of the table, so that weights lie in [0, 1]. */
void om_optics_radiance(om_optics *o, const double *s12, int n, const double L[3], const double *pol)
{
    free(o->rad);
    o->rad = (double *)malloc((size_t)n * 2 * sizeof(double));
    memcpy(o->rad, s12, (size_t)n * 2 * sizeof(double));
    o->n_rad = n;
    o->rad_mode = pol ? 2 : 1;
    o->rad_max = 0.0;
    for (int i = 0; i < 2 * n; ++i) if (s12[i] > o->rad_max) o->rad_max = s12[i];
    for (int a = 0; a < 3; ++a) { o->L[a] = L[a]; o->pol[a] = pol ? pol[a] : 0.0; }
}

double om_radiance(const om_optics *o, const double d0[3])
{
    if (!o->rad_mode) return 1.0;
    double c = d0[0] * o->L[0] + d0[1] * o->L[1] + d0[2] * o->L[2];
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double t = acos(c) / M_PI * (double)(o->n_rad - 1);
    int i = (int)floor(t);
    if (i > o->n_rad - 2) i = o->n_rad - 2;
    double f = t - (double)i;
    double s1 = (1.0 - f) * o->rad[2 * i] + f * o->rad[2 * i + 2];
    double s2 = (1.0 - f) * o->rad[2 * i + 1] + f * o->rad[2 * i + 3];
    double I_ = 0.5 * (s1 + s2);
    if (o->rad_mode == 2) {
        /* the scattering plane holds L and d0; the incident field's
         * component in it is along e = d0 - (d0.L) L */
        double e[3], e2 = 0.0, pe = 0.0;
        for (int a = 0; a < 3; ++a) { e[a] = d0[a] - c * o->L[a]; e2 += e[a] * e[a]; pe += o->pol[a] * e[a]; }
        double c2 = e2 > 0.0 ? pe * pe / e2 : 0.5;
        I_ = s2 * c2 + s1 * (1.0 - c2);
    }
    return I_ / o->rad_max;
}

/* the radiance weight of ray ray_id of a source (for tests) */
double om_ray_weight(const om_optics *o, const double src[3], uint64_t seed, uint32_t source_id, uint32_t ray_id,
                     uint32_t frame)
{
    double p[3], d[3], L2 = 0.0;
    om_lens_point(seed, source_id, ray_id, frame, o->aim_r, o->aim_z, p);
    for (int a = 0; a < 3; ++a) { d[a] = p[a] - src[a]; L2 += d[a] * d[a]; }
    double L = sqrt(L2);
    for (int a = 0; a < 3; ++a) d[a] /= L;
    return om_radiance(o, d);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 deposit: Gaussian spot of standard deviation sigma centred on the */
/* hit, integrated over each pixel with erf, over the pixels within 3 sigma  */
/* (clipped to the sensor), renormalised over that window and quantised to   */
/* 32.32 fixed point; the rounding remainder goes to the largest weight      */
/* (first in row-major order) so every ray adds exactly 2^32.               */
/* ------------------------------------------------------------------------ */
static void om_axis_weights(double p, double sp, int N, int *lo, int *hi, double *w /* size >= hi-lo+1 */)
{
    int a = (int)floor(p - 3.0 * sp);
    int b = (int)floor(p + 3.0 * sp);
    if (a < 0) a = 0;
    if (b > N - 1) b = N - 1;
    double s = 0.0;
    for (int i = a; i <= b; ++i) {
        double e1 = erf(((double)(i + 1) - p) / (M_SQRT2 * sp));
        double e0 = erf(((double)i - p) / (M_SQRT2 * sp));
        w[i - a] = 0.5 * (e1 - e0);
        s += w[i - a];
    }
    for (int i = a; i <= b; ++i) w[i - a] /= s;
    *lo = a; *hi = b;
}

/* returns the number of pixels touched; adds into image (row-major, y = row) */
/* A ray of radiance weight w (Sec. 3.1; 1 without Mie radiance) deposits
 * round(w 2^32) in all: each pixel's share w_i w_j w 2^32 rounded, the
 * remainder on the largest. */
int om_deposit_weighted(const om_optics *o, double px, double py, double w, int64_t *image, int atomic);

int om_deposit(const om_optics *o, double px, double py, int64_t *image, int atomic)
{
    return om_deposit_weighted(o, px, py, 1.0, image, atomic);
}

int om_deposit_weighted(const om_optics *o, double px, double py, double w, int64_t *image, int atomic)
{
    double sp = o->sigma / o->pitch;
    int xlo, xhi, ylo, yhi;
    double wx[4096], wy[4096];
    om_axis_weights(px, sp, o->W, &xlo, &xhi, wx);
    om_axis_weights(py, sp, o->H, &ylo, &yhi, wy);
    const double two32 = 4294967296.0 * w;
    int64_t sum = 0, qmax = -1;
    int imax = 0, jmax = 0;
    for (int j = ylo; j <= yhi; ++j)
        for (int i = xlo; i <= xhi; ++i) {
            int64_t q = (int64_t)llrint(wx[i - xlo] * wy[j - ylo] * two32);
            sum += q;
            if (q > qmax) { qmax = q; imax = i; jmax = j; }
        }
    int64_t rem = (int64_t)llrint(w * 4294967296.0) - sum;
    for (int j = ylo; j <= yhi; ++j)
        for (int i = xlo; i <= xhi; ++i) {
            int64_t q = (int64_t)llrint(wx[i - xlo] * wy[j - ylo] * two32);
            if (i == imax && j == jmax) q += rem;
            if (q == 0) continue;
            int64_t *dst = &image[(size_t)j * (size_t)o->W + (size_t)i];
            if (atomic) {
#pragma omp atomic
                *dst += q;
            } else {
                *dst += q;
            }
        }
    return (xhi - xlo + 1) * (yhi - ylo + 1);
}

/* ------------------------------------------------------------------------ */
/* Whole render: every ray of every source, image accumulated.  stats[6]    */
/* counts rays by final status.  Rays are independent (Sec. 3.5), so the    */
/* loop is spread over host threads; the integer image makes the order      */
/* irrelevant.                                                              */
/* ------------------------------------------------------------------------ */
void om_render(const om_medium *m, const om_optics *o, const double *sources, int64_t n_sources,
               int32_t rays_per_source, int64_t first_ray, int64_t ray_count,
               uint64_t seed, uint32_t frame, int integrator, double step,
               int64_t *image, int64_t *stats, int nthreads)
{
    int64_t total = n_sources * (int64_t)rays_per_source;
    int64_t end = first_ray + ray_count;
    if (end > total) end = total;
    int64_t cnt[6] = { 0, 0, 0, 0, 0, 0 };
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        int64_t lc[6] = { 0, 0, 0, 0, 0, 0 };
#pragma omp for schedule(dynamic, 256)
        for (int64_t r = first_ray; r < end; ++r) {
            int64_t s = r / rays_per_source;
            uint32_t k = (uint32_t)(r % rays_per_source);
            om_ray_state st;
            int status = om_trace(m, o, &sources[3 * s], seed, (uint32_t)s, k, frame, integrator, step, &st);
            if (status == OM_REACHED) {
                double w = o->rad_mode ? om_ray_weight(o, &sources[3 * s], seed, (uint32_t)s, k, frame) : 1.0;
                om_deposit_weighted(o, st.sensor_xy[0], st.sensor_xy[1], w, image, 1);
            }
            lc[status] += 1;
        }
#pragma omp critical
        for (int q = 0; q < 6; ++q) cnt[q] += lc[q];
    }
    if (stats) for (int q = 0; q < 6; ++q) stats[q] += cnt[q];
}

/* Per-ray states for a list of ray ids (id = source * rays_per_source + ray). */
void om_trace_many(const om_medium *m, const om_optics *o, const double *sources,
                   int32_t rays_per_source, const int64_t *ray_ids, int64_t n,
                   uint64_t seed, uint32_t frame, int integrator, double step,
                   om_ray_state *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        int64_t r = ray_ids[q];
        int64_t s = r / rays_per_source;
        uint32_t k = (uint32_t)(r % rays_per_source);
        om_trace(m, o, &sources[3 * s], seed, (uint32_t)s, k, frame, integrator, step, &out[q]);
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 9 (Sec. 4): the BOS theory deflection needs the integral over depth  */
/* of the transverse gradient of n, Delta X = (M Z_D / n0) * int grad n dz.  */
/* Reading: the integral runs along the straight line from a dot s toward   */
/* the point c (the centre of the lens), over the part of that line inside  */
/* the density box and between s and c, of the trilinearly sampled dn/dx    */
/* and dn/dy (the same samples the tracer uses), with respect to z.         */
/* Between two consecutive crossings of node planes the sample is a         */
/* product of three linear functions of z, a cubic; each such piece is      */
/* integrated with three-point Gauss-Legendre quadrature, which is exact    */
/* for polynomials of degree five or less.  Returns the number of pieces    */
/* (0: the line misses the box; -1: the line is parallel to the sensor).    */
/* ------------------------------------------------------------------------ */
static int om_cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int om_line_gradient_integral(const om_medium *m, const double s[3], const double c[3], double out[2])
{
    out[0] = 0.0;
    out[1] = 0.0;
    if (c[2] == s[2]) return -1;
    /* x(z) = s_x + a_x (z - s_z), y(z) = s_y + a_y (z - s_z) */
    double a[3];
    a[0] = (c[0] - s[0]) / (c[2] - s[2]);
    a[1] = (c[1] - s[1]) / (c[2] - s[2]);
    a[2] = 1.0;
    double z0 = fmin(s[2], c[2]), z1 = fmax(s[2], c[2]);
    for (int ax = 0; ax < 3; ++ax) {
        double lo = m->origin[ax], hi = m->origin[ax] + (double)(m->n[ax] - 1) * m->spacing[ax];
        if (a[ax] == 0.0) {
            if (s[ax] < lo || s[ax] > hi) return 0;
            continue;
        }
        /* z where coordinate ax equals lo and hi */
        double za = s[2] + (lo - s[ax]) / a[ax];
        double zb = s[2] + (hi - s[ax]) / a[ax];
        z0 = fmax(z0, fmin(za, zb));
        z1 = fmin(z1, fmax(za, zb));
    }
    if (!(z1 > z0)) return 0;
    /* breakpoints: the ends and every crossing of a node plane in between */
    int cap = 2 + m->n[0] + m->n[1] + m->n[2];
    double *zs = (double *)malloc((size_t)cap * sizeof(double));
    int nz = 0;
    zs[nz++] = z0;
    zs[nz++] = z1;
    for (int ax = 0; ax < 3; ++ax) {
        if (a[ax] == 0.0) continue;
        for (int i = 0; i < m->n[ax]; ++i) {
            double plane = m->origin[ax] + (double)i * m->spacing[ax];
            double zc = s[2] + (plane - s[ax]) / a[ax];
            if (zc > z0 && zc < z1) zs[nz++] = zc;
        }
    }
    qsort(zs, (size_t)nz, sizeof(double), om_cmp_double);
    const double xg[3] = { -sqrt(0.6), 0.0, sqrt(0.6) };
    const double wg[3] = { 5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0 };
    int pieces = 0;
    for (int q = 0; q + 1 < nz; ++q) {
        double za = zs[q], zb = zs[q + 1];
        if (!(zb > za)) continue;
        double mid = 0.5 * (za + zb), half = 0.5 * (zb - za);
        for (int g = 0; g < 3; ++g) {
            double z = mid + half * xg[g];
            double R[3] = { s[0] + a[0] * (z - s[2]), s[1] + a[1] * (z - s[2]), z };
            double dn, gr[3];
            om_sample(m, R, &dn, gr);
            out[0] += half * wg[g] * gr[0];
            out[1] += half * wg[g] * gr[1];
        }
        ++pieces;
    }
    free(zs);
    return pieces;
}

/* ------------------------------------------------------------------------ */
/* Image pairs for displacement analysis: the second frame's particles are  */
/* the first frame's moved by a velocity field u (3 components per node on  */
/* a grid like the density's, trilinear, clamped to the grid) over dt with   */
/* the explicit midpoint rule: k = u(x), x' = x + dt u(x + dt k / 2).        */
/* vel: [nz][ny][nx][3] float32.                                             */
/* ------------------------------------------------------------------------ */
static void om_vel_sample(const float *vel, const int n[3], const double o[3], const double h[3],
                          const double x[3], double u[3])
{
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double g = (x[a] - o[a]) / h[a];
        if (g < 0.0) g = 0.0;
        if (g > (double)(n[a] - 1)) g = (double)(n[a] - 1);
        int i = (int)floor(g);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = g - (double)i;
    }
    u[0] = u[1] = u[2] = 0.0;
    for (int c = 0; c < 8; ++c) {
        int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
        size_t p = (((size_t)(i0[2] + dk) * (size_t)n[1] + (size_t)(i0[1] + dj)) * (size_t)n[0] + (size_t)(i0[0] + di));
        for (int a = 0; a < 3; ++a) u[a] += w * (double)vel[3 * p + a];
    }
}

void om_advect(const double *src, int64_t n_src, const float *vel, int nx, int ny, int nz, const double origin[3],
               const double spacing[3], double dt, double *out)
{
    const int n[3] = { nx, ny, nz };
    for (int64_t q = 0; q < n_src; ++q) {
        const double *x = &src[3 * q];
        double k[3], xm[3], u[3];
        om_vel_sample(vel, n, origin, spacing, x, k);
        for (int a = 0; a < 3; ++a) xm[a] = x[a] + 0.5 * dt * k[a];
        om_vel_sample(vel, n, origin, spacing, xm, u);
        for (int a = 0; a < 3; ++a) out[3 * q + a] = x[a] + dt * u[a];
    }
}

/* 16-bit image (Sec. 3.4: about 1e4 rays per particle give a 16-bit
 * dynamic range): one count is d = llround(full_scale 2^32 / 65535) units of
 * the 32.32 image (full_scale rays read 65535); counts = the image divided
 * by d, rounded half up, clipped to [0, 65535] -- integer arithmetic once d
 * is fixed. */
void om_image_u16(const int64_t *image, int64_t n, double full_scale, uint16_t *out)
{
    int64_t d = (int64_t)llround(full_scale * 4294967296.0 / 65535.0);
    if (d < 1) d = 1;
    for (int64_t q = 0; q < n; ++q) {
        int64_t v = image[q] < 0 ? 0 : image[q];
        /* (v + floor(d/2)) / d, computed without overflow */
        int64_t c = v / d + ((v % d) >= d - d / 2 ? 1 : 0);
        out[q] = (uint16_t)(c > 65535 ? 65535 : c);
    }
}

/* helpers exposed for tests */
void om_sample_many(const om_medium *m, const double *x, int64_t n, double *dn, double *g)
{
    for (int64_t q = 0; q < n; ++q) om_sample(m, &x[3 * q], &dn[q], &g[3 * q]);
}

int om_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
