// Variable-h neighbour lists over the multi-level cell grid.
//
// N(i) = { j : |r_i - r_j|^2 < (3 max(h_i, h_j))^2 } with minimum-image
// separations on periodic axes and i itself included: every j for which a
// kernel W(r_ij, h_i), W(r_ij, h_j) or W(r_ij, h_ij) of the paper's gather
// sums (section 2) is non-zero.  Membership is decided by the FP64
// predicate with explicit round-to-nearest operations, so the sets are
// exactly those of the definition.
//
// Search: a particle of level l has 3h <= c_l.  Particle i visits only its
// own level and the coarser ones; there every neighbour lies within
// c_l >= 3 max(h_i, h_j) of i, i.e. in the 3x3 cells around it.  A pair
// whose j is coarser than i is found once, by i, and also written into
// j's list ("reverse" entries), so no particle ever scans the many cells of
// a finer level.
//
// Mixed path filter: each particle also carries FP32 coordinates relative
// to a global anchor lattice (cell side A ~ c0, integer anchor indices).
// The separation rebuilt from them has an absolute error far below the
// band used here; candidates inside the band around the support radius
// are re-tested with the FP64 predicate, so both paths give the same sets.
#pragma once

#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ bool table_lookup(const Grid &g, uint64_t key,
                                             uint32_t &s, uint32_t &e) {
    uint32_t slot = hash_slot(key, g.tmask);
    for (uint32_t it = 0; it <= g.tmask; ++it) {
        uint64_t t = __ldg(&g.tkey[slot]);
        if (t == key) {
            s = __ldg(&g.tstart[slot]);
            e = __ldg(&g.tend[slot]);
            return true;
        }
        if (t == EMPTY_KEY) return false;
        slot = (slot + 1) & g.tmask;
    }
    return false;
}

// Cell index ranges on one axis of one level for the query interval
// [x - Q, x + Q], clipped to the level's occupied bounding box [b0, b1].
// On a periodic axis the interval is cut into pieces that each map into
// [b0, b1] by one shift of the period; r[k] = {first, last, shift} with
// cell index = c + shift.  Returns the number of pieces (0..3).
struct AxisPieces {
    int first[3], last[3], shift[3];
    int n;
};

__device__ __forceinline__ void axis_pieces(const Domain &d, const Level &L,
                                            const int *bb, int ax, double x,
                                            double Q, AxisPieces &r) {
    const int nc = L.n[ax];
    const int b0 = __ldg(&bb[2 * ax]), b1 = __ldg(&bb[2 * ax + 1]);
    double lo = __ddiv_rn(__dsub_rn(__dsub_rn(x, Q), d.lo[ax]), L.w[ax]);
    double hi = __ddiv_rn(__dsub_rn(__dadd_rn(x, Q), d.lo[ax]), L.w[ax]);
    double flo = floor(lo), fhi = floor(hi);
    r.n = 0;
    if (d.periodic[ax]) {
        if (fhi - flo + 1.0 >= (double)nc) {
            r.first[0] = b0;
            r.last[0] = b1;
            r.shift[0] = 0;
            r.n = 1;
            return;
        }
        const int a0 = (int)flo, a1 = (int)fhi;
        for (int k = -1; k <= 1; ++k) {
            const int lo_k = max(a0, b0 + k * nc), hi_k = min(a1, b1 + k * nc);
            if (lo_k <= hi_k) {
                r.first[r.n] = lo_k;
                r.last[r.n] = hi_k;
                r.shift[r.n] = -k * nc;
                r.n++;
            }
        }
    } else {
        const int a0 = flo < (double)b0 ? b0 : (int)flo;
        const int a1 = fhi > (double)b1 ? b1 : (int)fhi;
        if (a0 <= a1) {
            r.first[0] = a0;
            r.last[0] = a1;
            r.shift[0] = 0;
            r.n = 1;
        }
    }
}

// Calls f(j) for every particle j in the cells of levels >= li that
// intersect the square of half side max(3 h_i, c_l) around (xi, yi).
template <class F>
__device__ __forceinline__ void for_each_candidate(const Grid &g,
                                                   const Domain &d, int li,
                                                   double xi, double yi,
                                                   double hi, F &&f) {
    const double Ri = __dmul_rn(3.0, hi);
    const uint32_t mask = g.level_mask & ~((1u << li) - 1u);
    for (uint32_t mm = mask; mm; mm &= mm - 1) {
        const int l = __ffs(mm) - 1;
        const int *bb = g.bbox + 4 * l;
        if (__ldg(&bb[0]) > __ldg(&bb[1])) continue;   // level holds no particle
        const Level &L = g.lev[l];
        // margin covers rounding in level and cell assignment
        const double Q = fmax(Ri, L.c) * (1.0 + 1e-7);
        AxisPieces px, py;
        axis_pieces(d, L, bb, 0, xi, Q, px);
        if (px.n == 0) continue;
        axis_pieces(d, L, bb, 1, yi, Q, py);
        const uint64_t lbits = (uint64_t)l << (2 * g.mbits);
        for (int ky = 0; ky < py.n; ++ky) {
            for (int cy = py.first[ky]; cy <= py.last[ky]; ++cy) {
                const uint64_t my = spread2((uint64_t)(cy + py.shift[ky])) << 1;
                for (int kx = 0; kx < px.n; ++kx) {
                    for (int cx = px.first[kx]; cx <= px.last[kx]; ++cx) {
                        uint32_t s, e;
                        if (!table_lookup(g, lbits | my |
                                                 spread2((uint64_t)(cx + px.shift[kx])),
                                          s, e))
                            continue;
                        for (uint32_t j = s; j < e; ++j) f((int)j);
                    }
                }
            }
        }
    }
}

// The FP64 neighbour predicate (definition above).
__device__ __forceinline__ bool pred_fp64(const Domain &d, double xi,
                                          double yi, double hi, double xj,
                                          double yj, double hj) {
    double dx = min_image(d, 0, __dsub_rn(xi, xj));
    double dy = min_image(d, 1, __dsub_rn(yi, yj));
    double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    double R = __dmul_rn(3.0, hi > hj ? hi : hj);
    return r2 < __dmul_rn(R, R);
}

// Anchor lattice for FP32 separations (mixed path).
struct Anchor {
    float A[2];      // anchor cell side per axis (float)
    int n[2];        // anchor cells per axis
    int periodic[2];
};

// FP32 separation r_i - r_j from anchor data: p = {xl, yl, h, gx|gy<<16}.
__device__ __forceinline__ void anchor_sep(const Anchor &an, const float4 &pi,
                                           const float4 &pj, float &dx,
                                           float &dy) {
    const unsigned gi = __float_as_uint(pi.w), gj = __float_as_uint(pj.w);
    int kx = (int)(gi & 0xffffu) - (int)(gj & 0xffffu);
    int ky = (int)(gi >> 16) - (int)(gj >> 16);
    if (an.periodic[0]) {
        if (2 * kx > an.n[0]) kx -= an.n[0];
        else if (2 * kx < -an.n[0]) kx += an.n[0];
    }
    if (an.periodic[1]) {
        if (2 * ky > an.n[1]) ky -= an.n[1];
        else if (2 * ky < -an.n[1]) ky += an.n[1];
    }
    dx = fmaf((float)kx, an.A[0], pi.x - pj.x);
    dy = fmaf((float)ky, an.A[1], pi.y - pj.y);
}

// Mixed-path predicate: FP32 test on anchor separations, FP64 predicate
// inside the uncertainty band.  The FP32 separation's absolute error is
// below (4 A + 2 |dx|) 2^-24 per axis (anchor offsets rounded to FP32, one
// FMA), so |r2_f - r2| < 2^-20 R (A + R) near r = R; the band is 2^-16 (R^2
// + 4 A R), a wide margin.  Returns membership and the FP32 separation.
__device__ __forceinline__ bool pred_mixed(const Domain &d, const Anchor &an,
                                           const float4 &pi, const float4 &pj,
                                           double xi, double yi, double hi,
                                           const double *__restrict__ x,
                                           const double *__restrict__ y,
                                           const double *__restrict__ h,
                                           int j, float &dx, float &dy,
                                           float &r2) {
    anchor_sep(an, pi, pj, dx, dy);
    r2 = fmaf(dx, dx, dy * dy);
    const float R = 3.0f * fmaxf(pi.z, pj.z);
    const float R2 = R * R;
    const float band = (R2 + 4.0f * fmaxf(an.A[0], an.A[1]) * R) *
                       (1.0f / 65536.0f);
    if (r2 < R2 - band) return true;
    if (r2 > R2 + band) return false;
    return pred_fp64(d, xi, yi, hi, __ldg(&x[j]), __ldg(&y[j]), __ldg(&h[j]));
}

}  // namespace sph
