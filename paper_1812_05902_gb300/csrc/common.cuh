// Internal types shared by the pivbos translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pivbos.h"

namespace pivbos {

// Device view of a medium: one float4 {n-1, dn/dx, dn/dy, dn/dz} per node,
// x fastest.  Grid coordinates g = (x - origin) / spacing.
struct DevMedium {
    const float4* field;
    int n[3];
    float h[3];          // spacing (float)
    float inv_h[3];      // 1 / spacing (float)
    double origin[3];
    double inv_hd[3];    // 1 / spacing (double)
    double lo[3], hi[3]; // box corners
    int max_steps;       // step budget for a parameter step of 1 m (scaled per render)
    int present;         // 0 = no medium: rays are straight everywhere
};

struct DevSurface {
    int type;
    int pad;
    double z, R, f, n_after, clear_r2;
};

struct DevOptics {
    int ns;
    int W, H;
    int pad;
    DevSurface s[PIVBOS_MAX_SURFACES];
    double n_object;
    double aim_z;
    double aim_r;
    float sigma_px;
    float pad2;        // spot sigma in pixels
    double sensor_z;
    double inv_pitch;
    double half_w, half_h; // W/2, H/2
    double win3;           // 3 sigma in pixels (double, for the window bounds)
    float inv_sqrt2_sigma; // 1 / (sqrt(2) sigma_px)
};

struct TraceParams {
    DevMedium m;
    DevOptics o;
    const double* sources;    // [S][3] device
    const uint32_t* perm;     // Morton order of sources (nullptr = identity)
    uint32_t n_sources;
    uint32_t rays_per_source;
    uint64_t seed;
    uint32_t frame;
    int max_steps;
    float step;               // parameter step
    double step_d;
    int* status_word;         // device status word (first error latched)
};

// Internal launchers (each defined in the translation unit holding the kernel).
cudaError_t launch_medium_prep(const float* rho, float4* field, int nx, int ny, int nz,
                               const double spacing[3], double K, cudaStream_t s);
cudaError_t launch_morton_sort(const double* sources, uint32_t n, uint64_t* keys_scratch,
                               uint32_t n_pow2, uint32_t* perm, cudaStream_t s);
cudaError_t launch_render(const TraceParams& p, int integrator, int64_t* image, int64_t* stats,
                          uint32_t rays_per_cta, cudaStream_t s);
cudaError_t launch_trace_states(const TraceParams& p, int integrator, const int64_t* ray_ids,
                                int64_t n_rays, pivbos_ray_state* out, cudaStream_t s);
cudaError_t launch_finalize(const int64_t* image, int64_t n, float* out, cudaStream_t s);

// Kernel timing hooks (api.cu): bracket a launch with events when enabled.
// Every launcher also counts its kernels (count_launches).
void timing_begin(const char* name, cudaStream_t s);
void count_launches(int64_t n);
void timing_end(const char* name, cudaStream_t s);

}  // namespace pivbos
