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
    const double *p, *ugx, *ugy;
};

// Calls f(k, dx, dy, r2) for every wall particle k with r_ik < 3 max(h_i,
// h_k) (the FP64 predicate), (dx, dy) = r_i - r_k by minimum image.
template <class F>
__device__ __forceinline__ void for_each_wall(const WallView &w,
                                              const Domain &d, double xi,
                                              double yi, double hi, F &&f) {
    if (w.n <= 0) return;
    for_each_candidate(w.g, d, 0, xi, yi, hi, [&](int k) {
        const double xk = __ldg(&w.x[k]), yk = __ldg(&w.y[k]);
        const double hk = __ldg(&w.h[k]);
        double dx = min_image(d, 0, __dsub_rn(xi, xk));
        double dy = min_image(d, 1, __dsub_rn(yi, yk));
        double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        double R = __dmul_rn(3.0, hi > hk ? hi : hk);
        if (r2 < __dmul_rn(R, R)) f(k, dx, dy, r2);
    });
}

struct WallBcArgs {
    WallView w;
    Grid g;                       // fluid cell structure
    Domain d;
    const double *x, *y, *h, *u, *v, *p;   // fluid
    double *pw, *ugx, *ugy;
};

void launch_wall_bc(cudaStream_t s, const WallBcArgs &a);

}  // namespace sph
