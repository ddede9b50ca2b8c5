// Thread teams: T consecutive threads of a warp (T = 1, 4 or 16) share one
// particle's neighbour work and combine their partial sums with shuffles.
// Small particle sets would otherwise leave most SMs idle with one thread
// per particle.  All shuffles and ballots use the team's own lane mask, so
// teams of one warp never wait on each other.
#pragma once

#include <cuda_runtime.h>

namespace sph {

template <int T>
struct Team {
    int lane;        // 0 .. T-1
    unsigned mask;   // this team's lanes within the warp
    __device__ __forceinline__ Team() {
        lane = threadIdx.x & (T - 1);
        const int wl = threadIdx.x & 31;
        mask = (T == 32) ? 0xffffffffu
                         : (((1u << T) - 1u) << (wl & ~(T - 1)));
    }
    __device__ __forceinline__ static int particle() {
        return (int)((blockIdx.x * blockDim.x + threadIdx.x) / T);
    }
};

template <int T, typename V>
__device__ __forceinline__ V team_sum(unsigned mask, V v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int T, typename V>
__device__ __forceinline__ V team_min(unsigned mask, V v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        V w = __shfl_xor_sync(mask, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Team size for n particles: enough threads to fill the GPU's 152 SMs a
// few times over, at most 16 lanes per particle.
inline int team_size(int n) {
    if (n <= 40000) return 16;
    if (n <= 300000) return 4;
    return 1;
}

}  // namespace sph
