// Internal types shared by the pivbos translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pivbos.h"

namespace pivbos {

// Double-float constant (hi + lo), prepared on the host.
struct dfc {
    float hi, lo;
};

// Device view of a medium: one float4 {n-1, dn/dx, dn/dy, dn/dz} per node,
// x fastest.  Grid coordinates g = (x - origin) / spacing.
struct DevMedium {
    const float4* field;
    int n[3];
    float h[3];          // spacing (float)
    float inv_h[3];      // 1 / spacing (float)
    dfc origin[3];       // node (0,0,0)
    dfc inv_hd[3];       // 1 / spacing (double-float)
    dfc lo[3], hi[3];    // box corners
    int max_steps;       // step budget for a parameter step of 1 m (scaled per render)
    int present;         // 0 = no medium: rays are straight everywhere
    float z_key;         // mid-plane of the box (ordering key plane)
};

struct DevSurface {
    int type;
    float R_f;         // signed radius (FP32, for sign tests)
    float clear_r2;    // clear radius squared (FP32, for the aperture tests)
    float pad;
    dfc z, R, invR;    // vertex position, radius, 1/R (lens array: pitch, 1/pitch)
    dfc eta, eta2;     // n_before / n_after and its square (refracting surfaces)
    dfc inv_f;         // 1 / focal length (ideal thin lens)
};

struct DevOptics {
    int ns;
    int W, H;
    float win3;            // 3 sigma in pixels
    DevSurface s[PIVBOS_MAX_SURFACES];
    dfc aim_z, aim_r;
    dfc sensor_z, inv_pitch;
    float half_w, half_h;  // W/2, H/2
    float inv_sqrt2_sigma; // 1 / (sqrt(2) sigma_px)
    float sigma_px;
    int tilted;            // 0: sensor square to the axis; 1: axes eu, ev and normal en below
    dfc eu[3], ev[3], en[3];
    // Mie radiance of the rays (Sec. 3.1): 0 none, 1 unpolarised, 2 polarised
    int rad_mode, rad_n;
    const float2* rad;     // |S1|^2, |S2|^2 over the table's maximum at rad_n angles 0..pi
    float rad_L[3];        // laser direction (unit)
    float rad_pol[3];      // polarisation (unit, normal to rad_L; mode 2)
};

// Whether optics hold a mirror, a lens array, a turned sensor or a radiance: the kernels
// compiled with the extended optics stage are launched only then.
inline bool optics_ext(const DevOptics& o)
{
    if (o.tilted || o.rad_mode) return true;
    for (int s = 0; s < o.ns; ++s)
        if (o.s[s].type == PIVBOS_SURF_MIRROR || o.s[s].type == PIVBOS_SURF_LENS_ARRAY) return true;
    return false;
}

struct TraceParams {
    DevMedium m;
    DevOptics o;
    const double* sources;    // [S][3] device (FP64 as given)
    const uint32_t* perm;     // Morton order of sources (nullptr = identity)
    const float2* src_df;     // [slot][3] sources in Morton order as double-float (render only)
    const uint32_t* ray_list; // render only the listed flat (slot, ray) indices (nullptr = all)
    uint32_t n_sources;
    uint32_t rays_per_source;
    uint32_t source_offset;   // global index of this call's first source (Philox counter)
    uint64_t seed;
    uint32_t frame;
    int max_steps;
    float step;               // parameter step
    double step_d;
    dfc step_df;
    int reorder;              // trace each CTA's rays in mid-plane Morton order
    int cell_cache;           // keep the last cell's corners in registers
    int* status_word;         // device status word (first error latched)
};

// One frame of a batch render (device copy).
struct BatchFrame {
    TraceParams p;
    int64_t* image;
    int64_t* stats;
    uint32_t rays_per_cta;
    uint32_t pad;
    uint64_t total_rays;
};

// Internal launchers (each defined in the translation unit holding the kernel).
cudaError_t launch_medium_prep(const float* rho, float4* field, int nx, int ny, int nz,
                               const double spacing[3], double K, cudaStream_t s);
// Sort the sources along a Morton curve: perm[slot] = source index, and
// src_df[3 * slot + a] = coordinate a of that source as double-float.
cudaError_t launch_morton_sort(const double* sources, uint32_t n, uint64_t* keys_scratch,
                               uint32_t n_pow2, uint32_t* perm, float2* src_df, cudaStream_t s);
cudaError_t launch_render(const TraceParams& p, int integrator, int64_t* image, int64_t* stats,
                          uint32_t rays_per_cta, cudaStream_t s);
cudaError_t launch_trace_states(const TraceParams& p, int integrator, const int64_t* ray_ids,
                                int64_t n_rays, pivbos_ray_state* out, cudaStream_t s);
// Render the rays listed in p.ray_list[0, min(*count, capacity)) (count on
// the device); persistent CTAs pop chunks of rays_per_cta list entries.
cudaError_t launch_list(const TraceParams& p, int integrator, const unsigned long long* count, uint32_t capacity,
                        int64_t* image, int64_t* stats, uint32_t rays_per_cta, unsigned long long* counter,
                        cudaStream_t s);
cudaError_t launch_batch(const BatchFrame* frames, const uint64_t* item_start, int n_frames, uint64_t total_items,
                         unsigned long long* counter, int integrator, bool cache, bool ext, int ctas_per_sm,
                         cudaStream_t s);

// Launch KERNEL_CALL(INTEG, CACHE, EXT) with the template arguments chosen
// at run time (integrator, cell cache, extended optics).
#define PV_DISPATCH(integrator, cache, ext, KERNEL_CALL)                                        \
    do {                                                                                       \
        if ((integrator) == PIVBOS_RK4) {                                                      \
            if (cache) { if (ext) KERNEL_CALL(PIVBOS_RK4, true, true); else KERNEL_CALL(PIVBOS_RK4, true, false); } \
            else { if (ext) KERNEL_CALL(PIVBOS_RK4, false, true); else KERNEL_CALL(PIVBOS_RK4, false, false); }   \
        } else {                                                                               \
            if (cache) { if (ext) KERNEL_CALL(PIVBOS_EULER, true, true); else KERNEL_CALL(PIVBOS_EULER, true, false); } \
            else { if (ext) KERNEL_CALL(PIVBOS_EULER, false, true); else KERNEL_CALL(PIVBOS_EULER, false, false); }   \
        }                                                                                      \
    } while (0)
cudaError_t launch_finalize(const int64_t* image, int64_t n, float* out, cudaStream_t s);

// Tuning knob (api.cu): keep cell corners in registers during integration;
// PIVBOS_CELL_CACHE=0/1 overrides the default (on for dense media).
int tuning_cell_cache(int dense);
// reorder / cell-cache choice for rendering through a medium (api.cu)
void choose_gather(const ::pivbos_medium* m, const ::pivbos_optics* o, double step, int integrator,
                   TraceParams& p);
// rays per CTA of a render (api.cu)
uint32_t rays_per_cta_setting(const TraceParams& p);

// Kernel timing hooks (api.cu): bracket a launch with events when enabled.
// Every launcher also counts its kernels (count_launches).
void timing_begin(const char* name, cudaStream_t s);
void count_launches(int64_t n);
void timing_end(const char* name, cudaStream_t s);

}  // namespace pivbos
