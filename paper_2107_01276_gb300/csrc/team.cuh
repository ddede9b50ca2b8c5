// Thread teams: T consecutive threads of a warp (T = 1, 4 or 16) share one
// particle's neighbour work and combine their partial sums with shuffles.
// Small particle sets would otherwise leave most SMs idle with one thread
// per particle.  All shuffles and ballots use the team's own lane mask, so
// teams of one warp never wait on each other.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

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

// Team size for n particles: a whole warp per particle while that still
// fits the GPU once (152 SMs x 64 resident warps), then 16 lanes while a
// team still fills it a few times over, 4 up to 300k, 1 beyond.
inline int team_size(int n) {
    if (n <= 152 * 64) return 32;
    if (n <= 40000) return 16;
    if (n <= 300000) return 4;
    return 1;
}

// Host-side dispatch: f(std::integral_constant<int, T>()) with T =
// team_size(n), or at least min_t (a power of two up to 32).
template <class F>
inline void with_team(int n, F &&f, int min_t = 1) {
    int t = team_size(n);
    if (t < min_t) t = min_t;
    switch (t) {
    case 32: f(std::integral_constant<int, 32>()); break;
    case 16: f(std::integral_constant<int, 16>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    default: f(std::integral_constant<int, 1>()); break;
    }
}

// f(std::integral_constant<int, T>()) with T = t when t is 1, 4, 16 or 32,
// else team_size(n).
template <class F>
inline void with_team_or(int t, int n, F &&f) {
    if (t != 1 && t != 4 && t != 16 && t != 32) t = team_size(n);
    switch (t) {
    case 32: f(std::integral_constant<int, 32>()); break;
    case 16: f(std::integral_constant<int, 16>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    default: f(std::integral_constant<int, 1>()); break;
    }
}

}  // namespace sph
