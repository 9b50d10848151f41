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
};

struct pivbos_optics {
    int device;
    pivbos::DevOptics d;
};

namespace pivbos {
// Message returned by pivbos_last_error() on this thread.
void set_last_error(const char* msg);
}  // namespace pivbos
