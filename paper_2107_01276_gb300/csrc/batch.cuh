// Work lists of the batched step: several independent simulations advance
// together, each per-particle phase (wall conditions, pass A, pass B, the
// PEC stages, the mid-step packing, the density store) and each kernel of
// a small set's neighbour build as one persistent launch over all of them.
// A work item is one block of one instance's single-launch grid; instance
// q owns items first[q] .. first[q + 1] - 1, and its argument block is
// args[q] in device memory.  The blocks of a launch step through the items
// with the grid's stride, so uneven instances share the SMs in proportion
// to their work.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sph {

struct BatchSpan {
    const int *first;   // k + 1 entries, first[0] = 0, first[k] = total
    int k;              // instances in this launch
    int total;          // work items
    // instance owning an item: the largest q with first[q] <= item
    __device__ __forceinline__ int find(int item) const {
        int lo = 0, hi = k;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&first[mid]) <= item)
                lo = mid;
            else
                hi = mid;
        }
        return lo;
    }
};

// One work item: its instance, and its block index within that
// instance's virtual grid (the grid a single-instance launch would use) of
// nvb blocks.
struct BatchItem {
    int q, vb, nvb;
};
__device__ __forceinline__ BatchItem batch_item(const BatchSpan &sp, int item) {
    BatchItem b;
    b.q = sp.find(item);
    const int f0 = __ldg(&sp.first[b.q]);
    b.vb = item - f0;
    b.nvb = __ldg(&sp.first[b.q + 1]) - f0;
    return b;
}

// Particles (or wall particles) one work item covers with teams of T
// threads in a 128-thread block.
constexpr int BATCH_THREADS = 128;
__host__ __device__ constexpr int batch_rows(int T) { return BATCH_THREADS / T; }

// Streaming multiprocessors of the current device (host).
int gpu_sms();

// Density store of the mixed path: rho (FP32) into the FP64 state.
struct RhoStoreArgs {
    int n;
    const float *src;
    double *dst;
};

}  // namespace sph
