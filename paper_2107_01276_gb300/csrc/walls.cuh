// Dummy wall particles seen from the fluid kernels (section 2.2).
#pragma once

#include "neighbors.cuh"
#include "sph_internal.cuh"

namespace sph {

// Walls sorted by their own cell keys; p, ugx, ugy from the wall BC;
// woff/wlist: for each fluid particle (current order) the walls within the
// reach of the last neighbour build, ascending (built by launch_wall_lists).
struct WallView {
    int n;
    Grid g;
    const double *x, *y, *h, *m, *uw, *vw;
    const float4 *pk;             // anchor coordinates of the walls
    const double *p, *ugx, *ugy;
    const uint32_t *woff, *wlist;
};

// Calls f(k, dx, dy, r2) for every wall particle k with r_ik < 3 max(h_i,
// h_k) (membership by the FP32 anchor filter with the FP64 predicate in
// its band), (dx, dy) = r_i - r_k by FP64 minimum image.  The candidates
// are fluid particle i's wall list of the last neighbour build (a
// superset: the walls within that build's reach), or without lists the
// cells of the wall grid around i; a team of T threads (lanes `mask`)
// takes every T-th candidate.  pi: particle i's anchor data.
template <int T, class F>
__device__ __forceinline__ void for_each_wall(const WallView &w, int i,
                                              const Domain &d,
                                              const Anchor &an,
                                              const float4 &pi, double xi,
                                              double yi, double hi, int lane,
                                              unsigned mask, F &&f) {
    if (w.n <= 0) return;
    if (!w.woff) {
        // no wall lists: walk the wall grid (cells looked up by the team)
        const float2 q = anchor_rel(an, pi);
        for_each_cell_team<T>(w.g, d, 0, q.x, q.y, pi.z, lane, mask,
                              [&](uint32_t s, uint32_t e) {
            for (uint32_t k = s + lane; k < e; k += T) {
                float fx, fy, fr2;
                if (!pred_mixed(d, an, pi, __ldg(&w.pk[k]), xi, yi, hi, w.x,
                                w.y, w.h, (int)k, fx, fy, fr2))
                    continue;
                const double dx = min_image(d, 0, __dsub_rn(xi, __ldg(&w.x[k])));
                const double dy = min_image(d, 1, __dsub_rn(yi, __ldg(&w.y[k])));
                f((int)k, dx, dy, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            }
        });
        return;
    }
    const uint32_t e = __ldg(&w.woff[i + 1]);
    for (uint32_t q = __ldg(&w.woff[i]) + lane; q < e; q += T) {
        const int k = (int)__ldg(&w.wlist[q]);
        float fx, fy, fr2;
        if (!pred_mixed(d, an, pi, __ldg(&w.pk[k]), xi, yi, hi, w.x, w.y,
                        w.h, k, fx, fy, fr2))
            continue;
        const double dx = min_image(d, 0, __dsub_rn(xi, __ldg(&w.x[k])));
        const double dy = min_image(d, 1, __dsub_rn(yi, __ldg(&w.y[k])));
        f(k, dx, dy, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    }
}

// Wall lists of the fluid particles, built from the walls' side: each wall
// particle walks the fluid grid (fine walls query few cells of every fluid
// level) and records itself for every fluid particle within reach, r <
// reach * 3 max(h_w, h_j) in FP32 anchor separations (reach >= 1.0001, far
// above the FP32 error: a superset of the exact sets while the particles
// move less than the build's skin).  Counting pass, scan, filling pass,
// then each list sorted (deterministic order).
struct WallListArgs {
    WallView w;
    Grid g;                       // fluid cell structure (fresh)
    Domain d;
    Anchor an;
    const float4 *pk;             // fluid anchor data
    float reach;
    uint32_t *cnt;                // n + 1 counts (zeroed by the build's key
                                  // and reset kernels)
    const uint32_t *off;          // n + 1 offsets (fill pass)
    uint32_t *cur;                // n cursors (zeroed likewise)
    uint32_t *list;
    uint32_t cap;
    int *overflow;
    uint32_t *longq, *nlong;      // segment-sort scratch (nlong zeroed)
};

// Counting pass and scan (off[n] = total entries); then the filling pass
// and the sort of each list.  n: fluid particles.
void launch_wall_lists_count(cudaStream_t s, int n, const WallListArgs &a,
                             SortScratch &sc, int *launches);
void launch_wall_lists_fill(cudaStream_t s, int n, const WallListArgs &a,
                            int *launches);

struct WallBcArgs {
    WallView w;
    Grid g;                       // fluid cell structure
    float qscale;                 // >= 1: the fluid moved since it was binned
    Domain d;
    Anchor an;
    const float4 *pk;             // fluid anchor data
    const double *x, *y, *h, *u, *v, *p;   // fluid
    double *pw, *ugx, *ugy;
};

void launch_wall_bc(cudaStream_t s, const WallBcArgs &a);

}  // namespace sph
