// Device-side bounds checks of a debug build (compiled with -DSPH_DEBUG).
// A failed check adds one to its translation unit's counter and the access
// it guards is skipped, never trapped: the context stays usable and the
// host reads the counts with sph_debug_failures.  Without SPH_DEBUG each
// check is the constant true and compiles away.
#pragma once

#include <cuda_runtime.h>

#ifdef SPH_DEBUG
static __device__ unsigned long long g_sph_debug_failures;
__device__ __forceinline__ bool sph_debug_check(bool ok) {
    if (!ok) atomicAdd(&g_sph_debug_failures, 1ull);
    return ok;
}
#define SPH_DCHECK(cond) sph_debug_check(cond)
// Host function `name`: the failures counted in this translation unit since
// its last call (the counter restarts at zero).
#define SPH_DEBUG_COUNTER(name)                                              \
    unsigned long long name() {                                              \
        unsigned long long v = 0, z = 0;                                     \
        cudaMemcpyFromSymbol(&v, g_sph_debug_failures, sizeof(v));           \
        cudaMemcpyToSymbol(g_sph_debug_failures, &z, sizeof(z));             \
        cudaGetLastError();                                                  \
        return v;                                                            \
    }
#else
#define SPH_DCHECK(cond) true
#define SPH_DEBUG_COUNTER(name) \
    unsigned long long name() { return 0; }
#endif
