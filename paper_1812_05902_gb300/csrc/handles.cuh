// Opaque handle layouts behind include/pivbos.h (library-internal).
#pragma once

#include "common.cuh"

struct pivbos_medium {
    int device;
    int n[3];
    double origin[3];
    double spacing[3];
    double K;
    float4* field;
    float* rho_scratch;   // device copy of host rho during a (re)fill
    uint64_t version = 0; // incremented by every refill (derived data, e.g. a surrogate, records it)
};

struct pivbos_optics {
    int device;
    pivbos::DevOptics d;
    double aim_z;          // creation arguments kept in FP64 (Eq. 9 theory, gather choice)
    double magnification;
    double n_object;
    double pixel_pitch;
    float2* rad_owned = nullptr;  // device radiance table this handle frees (d.rad), or NULL
};

namespace pivbos {
// Message returned by pivbos_last_error() on this thread.
void set_last_error(const char* msg);
// Validation and parameter assembly shared by every render entry point.
pivbos_status prepare_trace(const pivbos_medium* m, const pivbos_optics* o, const double* sources,
                            int64_t n_sources, int sources_on_device, int32_t rays_per_source, uint64_t seed,
                            uint32_t frame, int integrator, double step, TraceParams* p, int* dev, uint64_t* total);
// Device status word of device `dev` (a fixed device array; looked up once per device, never allocated).
pivbos_status device_status_word(int dev, int** out);
// Record a formatted message for pivbos_last_error() and return st.
pivbos_status failf(pivbos_status st, const char* fmt, ...);
// PIVBOS_OK for cudaSuccess; otherwise OOM or CUDA with a message naming `what`.
pivbos_status cuda_status(cudaError_t e, const char* what);
// A pointer declared as device memory must be device (or managed) memory of device `dev`.
pivbos_status device_pointer(const void* p, int dev, const char* what);
// Keep kernel timing out of captured streams.
void timing_suppress(bool on);
}  // namespace pivbos
