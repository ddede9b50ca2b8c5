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
                                             uint32_t &s, uint32_t &e,
                                             float *hmax = nullptr) {
    uint32_t slot = hash_slot(key, g.tmask);
    for (uint32_t it = 0; it <= g.tmask; ++it) {
        uint64_t t = __ldg(&g.tkey[slot]);
        if (t == key) {
            s = __ldg(&g.tstart[slot]);
            e = __ldg(&g.tend[slot]);
            if (hmax) *hmax = g.tmaxh ? __ldg(&g.tmaxh[slot]) : 3.0e38f;
            return true;
        }
        if (t == EMPTY_KEY) return false;
        slot = (slot + 1) & g.tmask;
    }
    return false;
}

// Pruning of the cells of a query.  gap2: squared distance from (xr, yr)
// to the rectangle of the cell (cx, cy) of level L, less a margin far
// above FP32 rounding.  On a periodic axis the distance is to the nearest
// periodic image of the cell (the indices may or may not be unwrapped);
// the edge cells of a non-periodic axis reach to infinity (particles
// outside the box are clamped into them).  A cell whose gap is at least the pair radius can hold no member:
// before the lookup the radius is qscale * max(3 h_i, c_l) (no particle of
// level l has 3h > c_l), after it qscale * 3 max(h_i, largest h of the
// cell).
__device__ __forceinline__ float cell_gap2(const Domain &d, const Level &L,
                                           int cx, int cy, float xr,
                                           float yr) {
    const int c[2] = {cx, cy};
    const float q[2] = {xr, yr};
    float g2 = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const float w = L.wf[ax];
        const float m = 1e-5f * (fabsf(q[ax]) + w);
        float gap;
        if (d.periodic[ax]) {
            const float P = (float)L.n[ax] * w;          // the period
            float t = q[ax] - ((float)c[ax] + 0.5f) * w;  // to the cell centre
            t -= P * rintf(t * L.invP[ax]);
            gap = fabsf(t) - 0.5f * w;
        } else {
            float lo = (float)c[ax] * w, hi = lo + w;
            if (c[ax] <= 0) lo = -3.0e38f;
            if (c[ax] >= L.n[ax] - 1) hi = 3.0e38f;
            gap = fmaxf(lo - q[ax], q[ax] - hi);
        }
        gap = fmaxf(0.0f, gap - m);
        g2 += gap * gap;
    }
    return g2;
}

// Lookup of cell (cx, cy) of level l (unwrapped indices, their periodic
// shifts sx, sy) with the two prunings above; false: nothing to visit.
__device__ __forceinline__ bool cell_visit(const Grid &g, const Domain &d,
                                           const Level &L, uint64_t lbits,
                                           int cx, int cy, int sx, int sy,
                                           float xr, float yr, float hi,
                                           float qscale, uint32_t &s,
                                           uint32_t &e) {
    const float g2 = cell_gap2(d, L, cx, cy, xr, yr);
    const float Rl = qscale * fmaxf(3.0f * hi, L.cf);
    if (g2 >= Rl * Rl) return false;
    float hmax;
    if (!table_lookup(g, lbits | (spread2((uint64_t)(cy + sy)) << 1) |
                             spread2((uint64_t)(cx + sx)),
                      s, e, &hmax))
        return false;
    const float Rc = qscale * 3.0f * fmaxf(hi, hmax);
    return g2 < Rc * Rc;
}

// Cell index ranges on one axis of one level for the query interval
// [x - Q, x + Q], clipped to the level's occupied bounding box [b0, b1].
// On a periodic axis the interval is cut into up to three pieces, one per
// period shift k = -1, 0, 1, that each map into [b0, b1]; piece k covers
// cells first[k]..last[k] (empty if first > last) with cell index c +
// shift[k].  Fixed slots keep the arrays in registers.
struct AxisPieces {
    int first[3], last[3], shift[3];
};

__device__ __forceinline__ bool axis_pieces(const Domain &d, const Level &L,
                                            const int *bb, int ax, float x,
                                            float Q, AxisPieces &r) {
    const int nc = L.n[ax];
    const int b0 = __ldg(&bb[2 * ax]), b1 = __ldg(&bb[2 * ax + 1]);
    // FP32 with a margin far above its rounding ((|x| + Q) / w 2^-21 cells):
    // the pieces only need to cover the exact cell range
    const float s = L.invw[ax];
    const float margin = (fabsf(x) + Q) * s * (1.0f / 1048576.0f) + (1.0f / 1024.0f);
    const float flo = floorf((x - Q) * s - margin);
    const float fhi = floorf((x + Q) * s + margin);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.first[k] = 1;
        r.last[k] = 0;
        r.shift[k] = 0;
    }
    if (d.periodic[ax]) {
        if (fhi - flo + 1.0f >= (float)nc) {
            r.first[1] = b0;
            r.last[1] = b1;
            return b0 <= b1;
        }
        const int a0 = (int)flo, a1 = (int)fhi;
        bool any = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int off = (k - 1) * nc;
            r.first[k] = max(a0, b0 + off);
            r.last[k] = min(a1, b1 + off);
            r.shift[k] = -off;
            any |= r.first[k] <= r.last[k];
        }
        return any;
    }
    r.first[1] = flo < (float)b0 ? b0 : (int)flo;
    r.last[1] = fhi > (float)b1 ? b1 : (int)fhi;
    return r.first[1] <= r.last[1];
}

// Whether the cells of a query (its axis pieces at level l) meet a block
// of the occupancy map holding particles; true without a map.
__device__ __forceinline__ bool occ_any(const Grid &g, int l, const int *bb,
                                        const AxisPieces &px,
                                        const AxisPieces &py) {
    if (!g.occ) return true;
    const int b0 = __ldg(&bb[0]), b1 = __ldg(&bb[1]);
    const int c0 = __ldg(&bb[2]), c1 = __ldg(&bb[3]);
    const uint32_t *o = g.occ + (size_t)l * OCC_N * (OCC_N / 32);
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
        if (px.first[kx] > px.last[kx]) continue;
        const int xlo = occ_block(px.first[kx] + px.shift[kx], b0, b1);
        const int xhi = occ_block(px.last[kx] + px.shift[kx], b0, b1);
        const uint64_t mx = (xhi >= 63 ? ~0ull : ((1ull << (xhi + 1)) - 1ull)) &
                            ~((1ull << xlo) - 1ull);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            if (py.first[ky] > py.last[ky]) continue;
            const int ylo = occ_block(py.first[ky] + py.shift[ky], c0, c1);
            const int yhi = occ_block(py.last[ky] + py.shift[ky], c0, c1);
            for (int by = ylo; by <= yhi; ++by) {
                const uint64_t row = (uint64_t)__ldg(&o[2 * by]) |
                                     ((uint64_t)__ldg(&o[2 * by + 1]) << 32);
                if (row & mx) return true;
            }
        }
    }
    return false;
}

// Calls f(s, e) for the particle range [s, e) of every occupied cell of
// levels >= li that intersects the square of half side max(3 h_i, c_l)
// around (xi, yi).  Cells come in a fixed order (level, then row, then
// column), so traversal order is deterministic.
// (xr, yr): position relative to the domain's lower corner, FP32.
//
// for_each_cell_scaled widens the square by qscale >= 1 (every pair with
// r_ij < qscale * 3 max(h_i, h_j) is then in the cells visited): the walk
// of lists with a skin.
template <class F>
__device__ __forceinline__ void for_each_cell_scaled(const Grid &g,
                                                     const Domain &d, int li,
                                                     float xr, float yr,
                                                     float hi, float qscale,
                                                     F &&f) {
    const float Ri = 3.0f * hi;
    const uint32_t mask = g.level_mask & ~((1u << li) - 1u);
    for (uint32_t mm = mask; mm; mm &= mm - 1) {
        const int l = __ffs(mm) - 1;
        const int *bb = g.bbox + 4 * l;
        if (__ldg(&bb[0]) > __ldg(&bb[1])) continue;   // level holds no particle
        const Level &L = g.lev[l];
        // margin covers rounding in level and cell assignment
        const float Q = qscale * fmaxf(Ri, L.cf) * (1.0f + 1e-5f);
        AxisPieces px, py;
        if (!axis_pieces(d, L, bb, 0, xr, Q, px)) continue;
        if (!axis_pieces(d, L, bb, 1, yr, Q, py)) continue;
        if (!occ_any(g, l, bb, px, py)) continue;   // no particle in reach
        const uint64_t lbits = (uint64_t)l << (2 * g.mbits);
        // piece loops unrolled so the piece arrays stay in registers
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            for (int cy = py.first[ky]; cy <= py.last[ky]; ++cy) {
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    for (int cx = px.first[kx]; cx <= px.last[kx]; ++cx) {
                        uint32_t s, e;
                        if (!cell_visit(g, d, L, lbits, cx, cy, px.shift[kx],
                                        py.shift[ky], xr, yr, hi, qscale, s, e))
                            continue;
                        f(s, e);
                    }
                }
            }
        }
    }
}

template <class F>
__device__ __forceinline__ void for_each_cell(const Grid &g, const Domain &d,
                                              int li, float xr, float yr,
                                              float hi, F &&f) {
    for_each_cell_scaled(g, d, li, xr, yr, hi, 1.0f, f);
}

// Team form of for_each_cell: the T lanes of a team (mask: the team's
// lanes) look up the cells of a level in parallel, lane t taking cells t,
// t + T, ..., and then every lane calls f(s, e) for the occupied cells in
// the same order as for_each_cell (level, then row, then column).  The
// hash lookups and cell arithmetic are thus done once per cell instead of
// once per lane; f may use team-wide shuffles and ballots.
template <int T, class F>
__device__ __forceinline__ void for_each_cell_team_scaled(
    const Grid &g, const Domain &d, int li, float xr, float yr, float hi,
    float qscale, int lane, unsigned mask, F &&f) {
    if constexpr (T == 1) {
        (void)lane;
        (void)mask;
        for_each_cell_scaled(g, d, li, xr, yr, hi, qscale, f);
        return;
    }
    const float Ri = 3.0f * hi;
    const uint32_t lmask = g.level_mask & ~((1u << li) - 1u);
    for (uint32_t mm = lmask; mm; mm &= mm - 1) {
        const int l = __ffs(mm) - 1;
        const int *bb = g.bbox + 4 * l;
        if (__ldg(&bb[0]) > __ldg(&bb[1])) continue;   // level holds no particle
        const Level &L = g.lev[l];
        const float Q = qscale * fmaxf(Ri, L.cf) * (1.0f + 1e-5f);
        AxisPieces px, py;
        if (!axis_pieces(d, L, bb, 0, xr, Q, px)) continue;
        if (!axis_pieces(d, L, bb, 1, yr, Q, py)) continue;
        if (!occ_any(g, l, bb, px, py)) continue;   // no particle in reach
        const int nx0 = max(0, px.last[0] - px.first[0] + 1);
        const int nx1 = max(0, px.last[1] - px.first[1] + 1);
        const int nx2 = max(0, px.last[2] - px.first[2] + 1);
        const int ny0 = max(0, py.last[0] - py.first[0] + 1);
        const int ny1 = max(0, py.last[1] - py.first[1] + 1);
        const int ny2 = max(0, py.last[2] - py.first[2] + 1);
        const int nx = nx0 + nx1 + nx2, ny = ny0 + ny1 + ny2;
        const int ncell = nx * ny;
        const uint64_t lbits = (uint64_t)l << (2 * g.mbits);
        for (int base = 0; base < ncell; base += T) {
            const int idx = base + lane;
            uint32_t s = 0, e = 0;
            if (idx < ncell) {
                const int iy = idx / nx, ix = idx - iy * nx;
                const int kx = ix < nx0 ? 0 : ix < nx0 + nx1 ? 1 : 2;
                const int ky = iy < ny0 ? 0 : iy < ny0 + ny1 ? 1 : 2;
                const int cx = kx == 0 ? px.first[0] + ix
                             : kx == 1 ? px.first[1] + (ix - nx0)
                                       : px.first[2] + (ix - nx0 - nx1);
                const int cy = ky == 0 ? py.first[0] + iy
                             : ky == 1 ? py.first[1] + (iy - ny0)
                                       : py.first[2] + (iy - ny0 - ny1);
                const int sx = kx == 0 ? px.shift[0] : kx == 1 ? px.shift[1] : px.shift[2];
                const int sy = ky == 0 ? py.shift[0] : ky == 1 ? py.shift[1] : py.shift[2];
                if (!cell_visit(g, d, L, lbits, cx, cy, sx, sy, xr, yr, hi,
                                qscale, s, e))
                    s = e = 0;
            }
            const int cnt = min(T, ncell - base);
            for (int t = 0; t < cnt; ++t) {
                const uint32_t ss = T == 1 ? s : __shfl_sync(mask, s, t, T);
                const uint32_t ee = T == 1 ? e : __shfl_sync(mask, e, t, T);
                if (ee > ss) f(ss, ee);
            }
        }
    }
}

// Candidate form of the team walk with one latency round per batch: for
// each level the lanes look up up to T cells at once, cell_ok(s, e) (called
// by the lane that found the cell) may drop a cell, and then the team's
// lanes take the candidates of all kept cells together, lane t the
// candidates t, t + T, ... of the concatenated ranges, located by a binary
// search over the lanes' running counts.  f(j) sees every candidate once,
// on one lane, with no order promised (for order-free reductions: minima,
// or sums whose rounding order may vary).  All lanes of the team execute
// the same iterations, so f and cell_ok may not use team shuffles.
//
// SYNC = true: f(j, valid) is called on every lane of the team in each
// batch iteration (valid false past the last candidate), so f may use team
// ballots; slot order is then the walk order (level, row, column, index),
// the candidates of one iteration being consecutive in it.
template <int T, bool SYNC = false, class CellOk, class F>
__device__ __forceinline__ void for_each_candidate_team(
    const Grid &g, const Domain &d, int li, float xr, float yr, float hi,
    float qscale, int lane, unsigned mask, CellOk &&cell_ok, F &&f) {
    if constexpr (T == 1) {
        (void)lane;
        (void)mask;
        for_each_cell_scaled(g, d, li, xr, yr, hi, qscale,
                             [&](uint32_t s, uint32_t e) {
            if (!cell_ok(s, e)) return;
            for (uint32_t j = s; j < e; ++j) {
                if constexpr (SYNC)
                    f(j, true);
                else
                    f(j);
            }
        });
        return;
    }
    const float Ri = 3.0f * hi;
    const uint32_t lmask = g.level_mask & ~((1u << li) - 1u);
    for (uint32_t mm = lmask; mm; mm &= mm - 1) {
        const int l = __ffs(mm) - 1;
        const int *bb = g.bbox + 4 * l;
        if (__ldg(&bb[0]) > __ldg(&bb[1])) continue;   // level holds no particle
        const Level &L = g.lev[l];
        const float Q = qscale * fmaxf(Ri, L.cf) * (1.0f + 1e-5f);
        AxisPieces px, py;
        if (!axis_pieces(d, L, bb, 0, xr, Q, px)) continue;
        if (!axis_pieces(d, L, bb, 1, yr, Q, py)) continue;
        if (!occ_any(g, l, bb, px, py)) continue;   // no particle in reach
        const int nx0 = max(0, px.last[0] - px.first[0] + 1);
        const int nx1 = max(0, px.last[1] - px.first[1] + 1);
        const int nx2 = max(0, px.last[2] - px.first[2] + 1);
        const int ny0 = max(0, py.last[0] - py.first[0] + 1);
        const int ny1 = max(0, py.last[1] - py.first[1] + 1);
        const int ny2 = max(0, py.last[2] - py.first[2] + 1);
        const int nx = nx0 + nx1 + nx2, ny = ny0 + ny1 + ny2;
        const int ncell = nx * ny;
        const uint64_t lbits = (uint64_t)l << (2 * g.mbits);
        for (int base = 0; base < ncell; base += T) {
            const int idx = base + lane;
            uint32_t s = 0, e = 0;
            if (idx < ncell) {
                const int iy = idx / nx, ix = idx - iy * nx;
                const int kx = ix < nx0 ? 0 : ix < nx0 + nx1 ? 1 : 2;
                const int ky = iy < ny0 ? 0 : iy < ny0 + ny1 ? 1 : 2;
                const int cx = kx == 0 ? px.first[0] + ix
                             : kx == 1 ? px.first[1] + (ix - nx0)
                                       : px.first[2] + (ix - nx0 - nx1);
                const int cy = ky == 0 ? py.first[0] + iy
                             : ky == 1 ? py.first[1] + (iy - ny0)
                                       : py.first[2] + (iy - ny0 - ny1);
                const int sx = kx == 0 ? px.shift[0] : kx == 1 ? px.shift[1] : px.shift[2];
                const int sy = ky == 0 ? py.shift[0] : ky == 1 ? py.shift[1] : py.shift[2];
                if (!cell_visit(g, d, L, lbits, cx, cy, sx, sy, xr, yr, hi,
                                qscale, s, e) ||
                    !(e > s && cell_ok(s, e)))
                    s = e = 0;
            }
            const uint32_t cnt = e - s;
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < T; o <<= 1) {
                const uint32_t t = __shfl_up_sync(mask, inc, o, T);
                if (lane >= o) inc += t;
            }
            const uint32_t total = __shfl_sync(mask, inc, T - 1, T);
            const uint32_t exc = inc - cnt;
            for (uint32_t q0 = 0; q0 < total; q0 += T) {
                const uint32_t q = q0 + (uint32_t)lane;
                const uint32_t qq = min(q, total - 1);
                int pos = 0;
#pragma unroll
                for (int st = T / 2; st; st >>= 1) {
                    const uint32_t v = __shfl_sync(mask, inc, pos + st - 1, T);
                    if (v <= qq) pos += st;
                }
                const uint32_t s0 = __shfl_sync(mask, s, pos, T);
                const uint32_t e0 = __shfl_sync(mask, exc, pos, T);
                if constexpr (SYNC)
                    f(s0 + (qq - e0), q < total);
                else if (q < total)
                    f(s0 + (qq - e0));
            }
        }
    }
}

template <int T, class F>
__device__ __forceinline__ void for_each_cell_team(const Grid &g,
                                                   const Domain &d, int li,
                                                   float xr, float yr,
                                                   float hi, int lane,
                                                   unsigned mask, F &&f) {
    for_each_cell_team_scaled<T>(g, d, li, xr, yr, hi, 1.0f, lane, mask, f);
}

// Calls f(j) for every particle j of the cells for_each_cell visits.
template <class F>
__device__ __forceinline__ void for_each_candidate(const Grid &g,
                                                   const Domain &d, int li,
                                                   float xr, float yr,
                                                   float hi, F &&f) {
    for_each_cell(g, d, li, xr, yr, hi, [&](uint32_t s, uint32_t e) {
        for (uint32_t j = s; j < e; ++j) f((int)j);
    });
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
    float iA[2];     // 1 / side, rounded to float
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

// Anchor record {xl, yl, h, gx | gy << 16} of a position: anchor cell g =
// floor((x - lo) / A) from the FP32 image of x - lo (clamped to the
// lattice; next to a cell edge it may be the neighbouring cell, which only
// moves the offset to within A / 256 outside [0, A): the separation error
// bound assumes an offset within about A) and the offset xl = x - lo - g A
// in FP64 with one rounding, then rounded to FP32.  One FP64 subtraction,
// one FMA and three conversions a coordinate (FP64 work is slow on this
// GPU).
__device__ __forceinline__ float4 anchor_record(double x, double y, double h,
                                                const double *lo,
                                                const double *A,
                                                const double *invA,
                                                const Anchor &an) {
    (void)invA;
    const double q[2] = {x, y};
    int g[2];
    float xl[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const double t = __dsub_rn(q[ax], lo[ax]);
        const float c = floorf((float)t * an.iA[ax]);
        const int gi = c < 0.0f ? 0 : (c > (float)(an.n[ax] - 1) ? an.n[ax] - 1 : (int)c);
        g[ax] = gi;
        xl[ax] = (float)__fma_rn(-(double)gi, A[ax], t);
    }
    return make_float4(xl[0], xl[1], (float)h,
                       __uint_as_float((unsigned)g[0] | ((unsigned)g[1] << 16)));
}

// Position relative to the domain's lower corner in FP32, from the anchor
// data p = {xl, yl, h, gx | gy << 16}.
__device__ __forceinline__ float2 anchor_rel(const Anchor &an, const float4 &p) {
    const unsigned g = __float_as_uint(p.w);
    return make_float2(fmaf((float)(g & 0xffffu), an.A[0], p.x),
                       fmaf((float)(g >> 16), an.A[1], p.y));
}

// Membership of a candidate whose FP32 anchor separation r2 is already
// known (hi, hj: the float h of the anchor records): the band test of
// pred_mixed, then the FP64 predicate inside the band.
__device__ __forceinline__ bool member_r2(const Domain &d, const Anchor &an,
                                          float r2, float hi, float hj,
                                          double xi, double yi, double hid,
                                          const double *__restrict__ x,
                                          const double *__restrict__ y,
                                          const double *__restrict__ h,
                                          int j) {
    const float R = 3.0f * fmaxf(hi, hj);
    const float R2 = R * R;
    const float band = (R2 + 4.0f * fmaxf(an.A[0], an.A[1]) * R) *
                       (1.0f / 65536.0f);
    if (r2 < R2 - band) return true;
    if (r2 > R2 + band) return false;
    return pred_fp64(d, xi, yi, hid, __ldg(&x[j]), __ldg(&y[j]), __ldg(&h[j]));
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
