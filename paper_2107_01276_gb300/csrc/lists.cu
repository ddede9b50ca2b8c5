// Per-rebuild packing (levels, FP32 anchor coordinates, float mirrors) and
// the CSR neighbour lists N(i) (definition and search in neighbors.cuh).
//
// List build: one walk per particle stages its own entries and counts the
// reverse ones -> exclusive scan -> place (own entries copied, reverse
// entries written into the coarser neighbours' lists) -> sort the reverse
// segment of each list, so lists are deterministic: own entries in
// traversal order, then the finer-level entries in ascending index.
#include "lists.cuh"
#include "neighbors.cuh"
#include "team.cuh"

#include <algorithm>

namespace sph {

// ------------------------------------------------------------------ pack --
__global__ void k_pack(PackArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.lev[i] = (uint8_t)(a.skey[i] >> a.lshift);
    const double x = a.x[i], y = a.y[i];
    int g[2];
    float xl[2];
    const double q[2] = {x, y};
    for (int ax = 0; ax < 2; ++ax) {
        double t = __dsub_rn(q[ax], a.lo[ax]);
        double c = floor(__ddiv_rn(t, a.Ad[ax]));
        int gi = c < 0.0 ? 0 : (c > (double)(a.an.n[ax] - 1) ? a.an.n[ax] - 1 : (int)c);
        g[ax] = gi;
        xl[ax] = (float)__dsub_rn(t, __dmul_rn((double)gi, a.Ad[ax]));
    }
    a.pk[i] = make_float4(xl[0], xl[1], (float)a.h[i],
                          __uint_as_float((unsigned)g[0] | ((unsigned)g[1] << 16)));
    if (a.tend) table_mark_end(i, a.n, a.skey, a.tkey, a.tend, a.tmask, a.h, a.tmaxh);
    if (!a.mixed) return;
    a.mf[i] = (float)a.m[i];
    a.pf[i] = (float)a.p[i];
    a.uf[i] = (float)a.u[i];
    a.vf[i] = (float)a.v[i];
}

// Anchor coordinates of a particle set (static sets: walls, background).
__global__ void k_anchor_pack(int n, const double *x, const double *y,
                              const double *h, double lo0, double lo1,
                              double A0, double A1, Anchor an, float4 *pk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double q[2] = {x[i], y[i]}, lo[2] = {lo0, lo1}, A[2] = {A0, A1};
    int g[2];
    float xl[2];
    for (int ax = 0; ax < 2; ++ax) {
        double t = __dsub_rn(q[ax], lo[ax]);
        double c = floor(__ddiv_rn(t, A[ax]));
        int gi = c < 0.0 ? 0 : (c > (double)(an.n[ax] - 1) ? an.n[ax] - 1 : (int)c);
        g[ax] = gi;
        xl[ax] = (float)__dsub_rn(t, __dmul_rn((double)gi, A[ax]));
    }
    pk[i] = make_float4(xl[0], xl[1], (float)h[i],
                        __uint_as_float((unsigned)g[0] | ((unsigned)g[1] << 16)));
}

// ------------------------------------------------------------ list build --
// Membership of candidate j for particle i: FP32 anchor filter with the
// FP64 predicate in its band (exact, for both precisions).
__device__ __forceinline__ bool member(const ListArgs &a, const float4 &pi,
                                       double xi, double yi, double hi,
                                       int j) {
    float dx, dy, r2;
    if (a.skin > 1.0f) {
        // skin lists: a superset is all that is needed, and the skin is far
        // wider than the FP32 error of the separation
        const float4 pj = __ldg(&a.pk[j]);
        anchor_sep(a.an, pi, pj, dx, dy);
        const float R = a.skin * 3.0f * fmaxf(pi.z, pj.z);
        return fmaf(dx, dx, dy * dy) < R * R;
    }
    return pred_mixed(a.d, a.an, pi, __ldg(&a.pk[j]), xi, yi, hi, a.x, a.y,
                      a.h, j, dx, dy, r2);
}

// Single-walk list build: a team of T lanes walks particle i's own and
// coarser levels (cells looked up in parallel, each cell's candidates
// taken T at a time, one per lane); the team's ballot orders each group,
// so own entries come in (cell, index) order whatever T is.  They go into
// a fixed-stride staging row of stage_w entries; particles with more own
// entries go to a queue that k_list_fill_queue handles with a second walk.

template <int T>
__global__ void __launch_bounds__(128) k_list_gather(ListArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const int li = a.lev[i];
    const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
    const float4 pi = a.pk[i];
    const float2 q = anchor_rel(a.an, pi);
    uint32_t k = 0;
    const uint32_t W = a.stage_w;
    uint32_t *row = a.stage + (size_t)i * W;
    const unsigned below = tm.mask & ((1u << (threadIdx.x & 31)) - 1u);
    for_each_cell_team_scaled<T>(a.g, a.d, li, q.x, q.y, pi.z, a.skin, tm.lane,
                                 tm.mask, [&](uint32_t s, uint32_t e) {
        for (uint32_t j0 = s; j0 < e; j0 += T) {
            const uint32_t j = j0 + tm.lane;
            const bool in = j < e && member(a, pi, xi, yi, hi, (int)j);
            const unsigned bal = T == 1 ? (in ? 1u : 0u)
                                        : __ballot_sync(tm.mask, in);
            if (in) {
                const uint32_t pos = k + (T == 1 ? 0u : __popc(bal & below));
                if (pos < W) row[pos] = j;
                if (__ldg(&a.lev[j]) > li) atomicAdd(&a.rev[j], 1u);
            }
            k += __popc(bal);
        }
    });
    if (tm.lane == 0) {
        a.own[i] = k;
        atomicMax(a.max_own, k);
        if (k > W) a.queue[atomicAdd(a.nqueue, 1u)] = (uint32_t)i;
    }
}

// Copies the staged own entries into place and writes the reverse entries
// (i into the list of each coarser neighbour j); T lanes per particle.
template <int T>
__global__ void __launch_bounds__(128) k_list_place(ListArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const uint32_t own = a.own[i];
    if (own <= a.stage_w) {               // else handled by k_list_fill_queue
        const int li = a.lev[i];
        const uint32_t base = a.off[i];
        const uint32_t *row = a.stage + (size_t)i * a.stage_w;
        const uint32_t cap = a.cap;
        for (uint32_t k = tm.lane; k < own; k += T) {
            const uint32_t j = row[k];
            if (base + k < cap) a.list[base + k] = j;
            if (__ldg(&a.lev[j]) > li) {
                const uint32_t rp = a.off[j] + a.own[j] + atomicAdd(&a.rev[j], 1u);
                if (rp < cap) a.list[rp] = (uint32_t)i;
            }
        }
    }
    if (i == a.n - 1 && tm.lane == 0 && a.off[a.n] > a.cap) atomicOr(a.overflow, 1);
}

__global__ void k_list_total(int n, const uint32_t *own, const uint32_t *rev,
                             uint32_t *tot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tot[i] = own[i] + rev[i];
}

// Second walk for the queued particles (more than stage_w own entries):
// same order as k_list_gather; teams take queue entries in turn.
template <int T>
__global__ void __launch_bounds__(128) k_list_fill_queue(ListArgs a) {
    const Team<T> tm;
    const uint32_t nq = *a.nqueue;
    const uint32_t team = (blockIdx.x * blockDim.x + threadIdx.x) / T;
    const uint32_t nteam = (gridDim.x * blockDim.x) / T;
    const unsigned below = tm.mask & ((1u << (threadIdx.x & 31)) - 1u);
    for (uint32_t qi = team; qi < nq; qi += nteam) {
        const int i = (int)a.queue[qi];
        const int li = a.lev[i];
        const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
        const float4 pi = a.pk[i];
        const float2 q = anchor_rel(a.an, pi);
        uint32_t k = a.off[i];
        const uint32_t cap = a.cap;
        for_each_cell_team_scaled<T>(a.g, a.d, li, q.x, q.y, pi.z, a.skin,
                                     tm.lane, tm.mask,
                                     [&](uint32_t s, uint32_t e) {
            for (uint32_t j0 = s; j0 < e; j0 += T) {
                const uint32_t j = j0 + tm.lane;
                const bool in = j < e && member(a, pi, xi, yi, hi, (int)j);
                const unsigned bal = __ballot_sync(tm.mask, in);
                if (in) {
                    const uint32_t pos = k + __popc(bal & below);
                    if (pos < cap) a.list[pos] = j;
                    if (__ldg(&a.lev[j]) > li) {
                        uint32_t rp = a.off[j] + a.own[j] + atomicAdd(&a.rev[j], 1u);
                        if (rp < cap) a.list[rp] = (uint32_t)i;
                    }
                }
                k += __popc(bal);
            }
        });
    }
}

// Sort of each reverse segment (ascending index).  Segments of at most 32
// entries (the common case: only particles next to a finer level have
// any) are sorted in registers by the particle's thread; longer ones are
// queued for a warp-wide bitonic sort in shared memory.
constexpr int SORT_REG = 32;
constexpr int SORT_SMEM = 1024;

__global__ void k_list_sort_rev(int n, const uint32_t *off, const uint32_t *own,
                                uint32_t *list, uint32_t cap, uint32_t *longq,
                                uint32_t *nlong) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t b = off[i] + own[i], e = off[i + 1];
    if (e > cap || e <= b + 1) return;
    const uint32_t len = e - b;
    if (len > SORT_REG) {
        longq[atomicAdd(nlong, 1u)] = (uint32_t)i;
        return;
    }
    uint32_t r[SORT_REG];
#pragma unroll
    for (int t = 0; t < SORT_REG; ++t) r[t] = t < (int)len ? list[b + t] : 0xffffffffu;
    // odd-even transposition sort, fixed indices (stays in registers)
#pragma unroll
    for (int round = 0; round < SORT_REG; ++round) {
#pragma unroll
        for (int t = round & 1; t + 1 < SORT_REG; t += 2) {
            uint32_t lo = min(r[t], r[t + 1]), hi = max(r[t], r[t + 1]);
            r[t] = lo;
            r[t + 1] = hi;
        }
    }
#pragma unroll
    for (int t = 0; t < SORT_REG; ++t)
        if (t < (int)len) list[b + t] = r[t];
}

__global__ void k_list_sort_long(const uint32_t *off, const uint32_t *own,
                                 uint32_t *list, const uint32_t *longq,
                                 const uint32_t *nlong) {
    __shared__ uint32_t buf[4][SORT_SMEM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *s = buf[w];
    const uint32_t nq = *nlong;
    const uint32_t gw = blockIdx.x * 4 + w, nw = gridDim.x * 4;
    for (uint32_t q = gw; q < nq; q += nw) {
        const uint32_t i = longq[q];
        const uint32_t b = off[i] + own[i], e = off[i + 1];
        const uint32_t len = e - b;
        if (len > SORT_SMEM) {
            // rare: plain insertion sort by one lane
            if (lane == 0) {
                for (uint32_t k = b + 1; k < e; ++k) {
                    uint32_t v = list[k], m = k;
                    while (m > b && list[m - 1] > v) {
                        list[m] = list[m - 1];
                        --m;
                    }
                    list[m] = v;
                }
            }
            __syncwarp();
            continue;
        }
        uint32_t P = 32;
        while (P < len) P <<= 1;
        for (uint32_t t = lane; t < P; t += 32) s[t] = t < len ? list[b + t] : 0xffffffffu;
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t t = lane; t < P; t += 32) {
                    uint32_t ixj = t ^ j;
                    if (ixj > t) {
                        uint32_t x0 = s[t], x1 = s[ixj];
                        bool asc = (t & k) == 0;
                        if ((x0 > x1) == asc) {
                            s[t] = x1;
                            s[ixj] = x0;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (uint32_t t = lane; t < len; t += 32) list[b + t] = s[t];
        __syncwarp();
    }
}

// ------------------------------------------------------------- launchers --
static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

void launch_pack(cudaStream_t s, const PackArgs &a) {
    if (a.n > 0) k_pack<<<nblk(a.n, 256), 256, 0, s>>>(a);
}
void launch_anchor_pack(cudaStream_t s, int n, const double *x,
                        const double *y, const double *h, const double *lo,
                        const double *A, const Anchor &an, float4 *pk) {
    if (n > 0)
        k_anchor_pack<<<nblk(n, 256), 256, 0, s>>>(n, x, y, h, lo[0], lo[1],
                                                    A[0], A[1], an, pk);
}

void launch_list_walk(cudaStream_t s, const ListArgs &a, int *launches) {
    const int n = a.n;
    if (n <= 0) return;
    with_team(n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_list_gather<T><<<nblk(n * T, 128), 128, 0, s>>>(a);
    });
    *launches += 1;
}

void list_offsets(cudaStream_t s, const ListArgs &a, SortScratch &sc,
                  uint32_t *tot_tmp, int *launches) {
    const int n = a.n;
    if (n <= 0) {
        cudaMemsetAsync(a.off, 0, sizeof(uint32_t), s);
        return;
    }
    if (list_offsets_small(s, a.own, a.rev, a.off, n, launches)) return;
    k_list_total<<<nblk(n, 256), 256, 0, s>>>(n, a.own, a.rev, tot_tmp);
    // off has n + 1 entries: scan n + 1 values with a trailing zero
    cudaMemsetAsync(tot_tmp + n, 0, sizeof(uint32_t), s);
    exclusive_scan(s, tot_tmp, a.off, n + 1, nullptr, sc, launches);
    cudaMemsetAsync(a.rev, 0, sizeof(uint32_t) * n, s);
    *launches += 1;
}

void build_lists_fill(cudaStream_t s, ListArgs a, bool mixed, bool queue,
                      int *launches) {
    (void)mixed;
    const int n = a.n;
    if (n <= 0) return;
    // at least 16 lanes per particle: a list's entries are then read from
    // the staging row and written to the list in 64-byte runs
    with_team(n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_list_place<T><<<nblk(n * T, 128), 128, 0, s>>>(a);
    }, 16);
    if (queue) k_list_fill_queue<16><<<152 * 4, 128, 0, s>>>(a);
    k_list_sort_rev<<<nblk(n, 256), 256, 0, s>>>(n, a.off, a.own, a.list, a.cap,
                                                  a.longq, a.nlong);
    // up to one warp per particle (4 per block): the long segments are
    // sorted in parallel whatever their number; idle warps exit at once
    k_list_sort_long<<<std::max(1, std::min(152 * 16, nblk(n, 4))), 128, 0, s>>>(
        a.off, a.own, a.list, a.longq, a.nlong);
    *launches += 4;
}

}  // namespace sph
