// Device checks of a loaded fluid set (load_check.cuh): one grid-stride
// pass over x, y, h, m and the ids, warp reductions, one atomic per warp.
#include <math.h>

#include <algorithm>

#include "batch.cuh"
#include "load_check.cuh"

namespace sph {

__global__ void k_load_check(long long n, const double *x, const double *y,
                             const double *h, const double *m,
                             const int64_t *id, Domain d, LoadCheckOut *out) {
    unsigned long long lo = ~0ull, hi = 0ull;
    long long imax = -1;
    int bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const double hi_ = h[i], mi = m[i];
        if (hi_ > 0.0 && isfinite(hi_) && mi > 0.0 && isfinite(mi)) {
            // positive doubles order as their bit patterns
            const unsigned long long b = (unsigned long long)__double_as_longlong(hi_);
            lo = b < lo ? b : lo;
            hi = b > hi ? b : hi;
        } else {
            bad |= LOAD_BAD_HM;
        }
        const double q[2] = {x[i], y[i]};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const bool in = d.periodic[a] ? (q[a] >= d.lo[a] && q[a] < d.hi[a])
                                          : (q[a] >= d.lo[a] && q[a] <= d.hi[a]);
            if (!in || !isfinite(q[a])) bad |= LOAD_BAD_POS;
        }
        if (id) imax = max(imax, (long long)id[i]);
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
        imax = max(imax, __shfl_xor_sync(0xffffffffu, imax, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo != ~0ull) atomicMin(&out->hmin, lo);
        if (hi != 0ull) atomicMax(&out->hmax, hi);
        if (imax >= 0) atomicMax(&out->idmax, imax);
        if (bad) atomicOr(&out->bad, bad);
    }
}

void launch_load_check(cudaStream_t s, long long n, const double *x,
                       const double *y, const double *h, const double *m,
                       const int64_t *id, const Domain &d, LoadCheckOut *out) {
    // hmin = all ones, hmax = 0, idmax = -1 (all ones), bad = 0
    cudaMemsetAsync(out, 0, sizeof(LoadCheckOut), s);
    cudaMemsetAsync(&out->hmin, 0xff, sizeof(unsigned long long), s);
    cudaMemsetAsync(&out->idmax, 0xff, sizeof(long long), s);
    if (n <= 0) return;
    const long long blocks = std::min<long long>((n + 255) / 256, 8ll * gpu_sms());
    k_load_check<<<(int)blocks, 256, 0, s>>>(n, x, y, h, m, id, d, out);
}

}  // namespace sph
