// Checks of a fluid set on the device as sph_load_particles receives it
// (include/sph.h): h and m positive and finite, positions finite and in
// the box, with the least and largest h and the largest id.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

enum : int {
    LOAD_BAD_HM = 1,    // an h or m not positive and finite
    LOAD_BAD_POS = 2,   // a position outside the box or not finite
};

struct LoadCheckOut {
    unsigned long long hmin, hmax;   // bit patterns of positive doubles
    long long idmax;                 // -1 without ids
    int bad;                         // LOAD_BAD_* bits
    int pad;
};

// id may be NULL.  out is reset on the stream first.
void launch_load_check(cudaStream_t s, long long n, const double *x,
                       const double *y, const double *h, const double *m,
                       const int64_t *id, const Domain &d, LoadCheckOut *out);

}  // namespace sph
