// Dummy wall particles seen from the fluid kernels (section 2.2).
#pragma once

#include "neighbors.cuh"
#include "sph_internal.cuh"

namespace sph {

// Walls sorted by their own cell keys; p, ugx, ugy from the wall BC.
struct WallView {
    int n;
    Grid g;
    const double *x, *y, *h, *m, *uw, *vw;
    const float4 *pk;             // anchor coordinates of the walls
    const double *p, *ugx, *ugy;
};

// Calls f(k, dx, dy, r2) for every wall particle k with r_ik < 3 max(h_i,
// h_k) (membership by the FP32 anchor filter with the FP64 predicate in
// its band), (dx, dy) = r_i - r_k by FP64 minimum image.  With a team of T
// threads (lanes `mask`), the team looks the wall cells up together and
// lane `lane` takes every T-th wall of each cell.  pi: particle i's anchor
// data.
template <int T, class F>
__device__ __forceinline__ void for_each_wall(const WallView &w,
                                              const Domain &d,
                                              const Anchor &an,
                                              const float4 &pi, double xi,
                                              double yi, double hi, int lane,
                                              unsigned mask, F &&f) {
    if (w.n <= 0) return;
    const float2 q = anchor_rel(an, pi);
    for_each_cell_team<T>(w.g, d, 0, q.x, q.y, pi.z, lane, mask,
                          [&](uint32_t s, uint32_t e) {
        for (uint32_t k = s + lane; k < e; k += T) {
            float fx, fy, fr2;
            if (!pred_mixed(d, an, pi, __ldg(&w.pk[k]), xi, yi, hi, w.x, w.y,
                            w.h, (int)k, fx, fy, fr2))
                continue;
            const double dx = min_image(d, 0, __dsub_rn(xi, __ldg(&w.x[k])));
            const double dy = min_image(d, 1, __dsub_rn(yi, __ldg(&w.y[k])));
            f((int)k, dx, dy, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        }
    });
}

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
