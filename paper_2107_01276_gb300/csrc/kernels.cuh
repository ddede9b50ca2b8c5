// Kernel function and pair separation shared by the pair kernels.
#pragma once

#include "neighbors.cuh"
#include "sph_internal.cuh"

namespace sph {

// Quintic spline in q (section 2, Eq. kernel) without sigma2, and its
// q-derivative, branch free: with a = max(3 - q, 0), b = max(2 - q, 0),
// c = max(1 - q, 0), w = a^5 - 6 b^5 + 15 c^5 and dw/dq = -5 a^4 + 30 b^4
// - 75 c^4 (every term vanishes where its base is clipped to zero).  The
// clip is one max instruction (a NaN q clips to zero).
// sigma2 = 7 / (478 pi h^2); dW/dr = sigma2 / h * dw(q).
__device__ __forceinline__ float clip0(float t) { return fmaxf(t, 0.0f); }
__device__ __forceinline__ double clip0(double t) { return fmax(t, 0.0); }

template <typename R>
__device__ __forceinline__ R qs_w(R q) {
    const R a = clip0(R(3) - q);
    const R b = clip0(R(2) - q);
    const R c = clip0(R(1) - q);
    const R a2 = a * a, b2 = b * b, c2 = c * c;
    return a2 * a2 * a - R(6) * (b2 * b2 * b) + R(15) * (c2 * c2 * c);
}

template <typename R>
__device__ __forceinline__ R qs_dw(R q) {
    const R a = clip0(R(3) - q);
    const R b = clip0(R(2) - q);
    const R c = clip0(R(1) - q);
    const R a2 = a * a, b2 = b * b, c2 = c * c;
    return R(-5) * (a2 * a2) + R(30) * (b2 * b2) - R(75) * (c2 * c2);
}

// a / b and 1/sqrt(x): IEEE in double; the fast FP32 forms (at most 2 ulp)
// in float, well inside the mixed path's tolerance.
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double frsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }

// Four values of one neighbour, loaded together.
template <typename R> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = double4_32a; };

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
    // with h_j (FP64 array)
    __device__ __forceinline__ void get(const Domain &d, const Anchor &an,
                                        const double *x, const double *y,
                                        const double *h, const float4 *pk,
                                        int j, double &dx, double &dy,
                                        double &r2, double &hj) const {
        get(d, an, x, y, pk, j, dx, dy, r2);
        hj = __ldg(&h[j]);
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
    // with h_j (from the anchor record)
    __device__ __forceinline__ void get(const Domain &, const Anchor &an,
                                        const double *, const double *,
                                        const double *, const float4 *pk,
                                        int j, float &dx, float &dy,
                                        float &r2, float &hj) const {
        const float4 pj = __ldg(&pk[j]);
        anchor_sep(an, pi, pj, dx, dy);
        r2 = fmaf(dx, dx, dy * dy);
        hj = pj.z;
    }
};


}  // namespace sph
