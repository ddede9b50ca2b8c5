// Kernel function and pair separation shared by the pair kernels.
#pragma once

#include "neighbors.cuh"
#include "sph_internal.cuh"

namespace sph {

// Quintic spline in q (section 2, Eq. kernel) without sigma2, and its
// q-derivative.  sigma2 = 7 / (478 pi h^2); dW/dr = sigma2 / h * dw(q).
template <typename R>
__device__ __forceinline__ R qs_w(R q) {
    if (q >= R(3)) return R(0);
    R a = R(3) - q, a2 = a * a;
    R w = a2 * a2 * a;
    if (q < R(2)) {
        R b = R(2) - q, b2 = b * b;
        w -= R(6) * (b2 * b2 * b);
        if (q < R(1)) {
            R c = R(1) - q, c2 = c * c;
            w += R(15) * (c2 * c2 * c);
        }
    }
    return w;
}

template <typename R>
__device__ __forceinline__ R qs_dw(R q) {
    if (q >= R(3)) return R(0);
    R a = R(3) - q, a2 = a * a;
    R w = R(-5) * (a2 * a2);
    if (q < R(2)) {
        R b = R(2) - q, b2 = b * b;
        w += R(30) * (b2 * b2);
        if (q < R(1)) {
            R c = R(1) - q, c2 = c * c;
            w -= R(75) * (c2 * c2);
        }
    }
    return w;
}

template <typename R>
__device__ __forceinline__ R sigma_norm() {
    return R(7.0 / (478.0 * PI));
}

// Separation r_i - r_j of list entry j: FP64 minimum image on the FP64
// path; on the mixed path rebuilt in FP32 from the anchor coordinates.
template <typename R> struct Sep;
template <> struct Sep<double> {
    double xi, yi;
    __device__ __forceinline__ void init(const Domain &, const double *x,
                                         const double *y, const float4 *, int i) {
        xi = x[i];
        yi = y[i];
    }
    __device__ __forceinline__ void get(const Domain &d, const Anchor &,
                                        const double *x, const double *y,
                                        const float4 *, int j, double &dx,
                                        double &dy, double &r2) const {
        dx = min_image(d, 0, __dsub_rn(xi, __ldg(&x[j])));
        dy = min_image(d, 1, __dsub_rn(yi, __ldg(&y[j])));
        r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    }
};
template <> struct Sep<float> {
    float4 pi;
    __device__ __forceinline__ void init(const Domain &, const double *,
                                         const double *, const float4 *pk, int i) {
        pi = pk[i];
    }
    __device__ __forceinline__ void get(const Domain &, const Anchor &an,
                                        const double *, const double *,
                                        const float4 *pk, int j, float &dx,
                                        float &dy, float &r2) const {
        anchor_sep(an, pi, __ldg(&pk[j]), dx, dy);
        r2 = fmaf(dx, dx, dy * dy);
    }
};


}  // namespace sph
