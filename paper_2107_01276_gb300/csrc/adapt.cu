// Adaptive refinement (section 3): resolution from the background,
// split, mutual-closest merge, shift with Taylor correction, h update.
// FP64 throughout, with explicitly rounded operations wherever a result
// feeds a decision (split test, merge admissibility and closest partner),
// so the decisions match the definition bit for bit.
#include "adapt.cuh"
#include "debug_checks.cuh"
#include "kernels.cuh"
#include "neighbors.cuh"
#include "team.cuh"

namespace sph {

// Quintic spline in FP64 with the operation order of its definition
// (section 2, Eq. kernel): sigma2 = 7 / (478 pi h^2), q = r / h.
__device__ __forceinline__ double p5_rn(double a) {
    return __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(a, a), a), a), a);
}
__device__ __forceinline__ double w_rn(double q) {
    if (q >= 3.0) return 0.0;
    double w = p5_rn(__dsub_rn(3.0, q));
    if (q < 2.0) w = __dsub_rn(w, __dmul_rn(6.0, p5_rn(__dsub_rn(2.0, q))));
    if (q < 1.0) w = __dadd_rn(w, __dmul_rn(15.0, p5_rn(__dsub_rn(1.0, q))));
    return w;
}
__device__ __forceinline__ double W_rn(double r, double h) {
    double s = __ddiv_rn(7.0, __dmul_rn(__dmul_rn(__dmul_rn(478.0, PI), h), h));
    return __dmul_rn(s, w_rn(__ddiv_rn(r, h)));
}
__device__ __forceinline__ double wrap_rn(const Domain &d, int a, double x) {
    if (d.periodic[a]) {
        if (x >= d.hi[a])
            x = __dsub_rn(x, d.L[a]);
        else if (x < d.lo[a])
            x = __dadd_rn(x, d.L[a]);
    }
    return x;
}

__device__ __forceinline__ void sep_rn(const Domain &d, double xi, double yi,
                                       double xj, double yj, double &dx,
                                       double &dy, double &r2) {
    dx = min_image(d, 0, __dsub_rn(xi, xj));
    dy = min_image(d, 1, __dsub_rn(yi, yj));
    r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// ------------------------------------------- resolution from background --
// m_ref,i = min rho0 ds_b^2 over background b with r_ib < 3 max(h_i, h_b)
// (section 3.3); particles with none in range are queued for the nearest
// background particle.  m_max = 1.05 m_ref, m_min = 0.5 m_ref.
template <int T>
__global__ void __launch_bounds__(128) k_bg_mref(BgArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
    const float4 pi = a.pk[i];
    const float2 q = anchor_rel(a.an, pi);
    double best = 1e308;
    // Levels come finest first, so the running minimum soon exceeds no
    // coarse cell's least m_ref: a cell whose least rho0 ds^2 is not below
    // the running minimum of the lane that looked it up is dropped (its
    // candidates cannot lower the team's minimum, which is at most that
    // lane's; rounding is monotone in ds).  best: the lane's own minimum
    // over the candidates it takes; the team's is taken at the end.
    for_each_candidate_team<T>(a.g, a.d, 0, q.x, q.y, pi.z, 1.0f, tm.lane,
                               tm.mask, [&](uint32_t s, uint32_t) {
        const double dmin = __ldg(&a.bcmin[s]);
        return __dmul_rn(__dmul_rn(a.rho0, dmin), dmin) < best;
    }, [&](uint32_t b) {
        float fx, fy, fr2;
        if (pred_mixed(a.d, a.an, pi, __ldg(&a.bpk[b]), xi, yi, hi, a.bx,
                       a.by, a.bh, (int)b, fx, fy, fr2)) {
            const double ds = __ldg(&a.bds[b]);
            const double mref = __dmul_rn(__dmul_rn(a.rho0, ds), ds);
            best = mref < best ? mref : best;
        }
    });
    best = team_min<T>(tm.mask, best);
    if (tm.lane != 0) return;
    if (best == 1e308) {
        a.queue[atomicAdd(a.nqueue, 1u)] = (uint32_t)i;
        return;
    }
    a.mmax[i] = __dmul_rn(1.05, best);
    a.mmin[i] = __dmul_rn(0.5, best);
}

// Nearest background particle (least r^2, then least load index) for the
// queued fluid particles; a warp per particle.
__global__ void k_bg_nearest(BgArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nq = *a.nqueue;
    for (uint32_t q = w; q < nq; q += nw) {
        const int i = (int)a.queue[q];
        const double xi = a.x[i], yi = a.y[i];
        double br2 = 1e308;
        long long bidx = -1;
        int bb = -1;
        for (int b = lane; b < a.nb; b += 32) {
            double dx, dy, r2;
            sep_rn(a.d, xi, yi, a.bx[b], a.by[b], dx, dy, r2);
            long long id = a.bid[b];
            if (r2 < br2 || (r2 == br2 && id < bidx)) {
                br2 = r2;
                bidx = id;
                bb = b;
            }
        }
        for (int o = 16; o; o >>= 1) {
            double r2o = __shfl_xor_sync(0xffffffffu, br2, o);
            long long ido = __shfl_xor_sync(0xffffffffu, bidx, o);
            int bo = __shfl_xor_sync(0xffffffffu, bb, o);
            if (bo >= 0 && (bb < 0 || r2o < br2 || (r2o == br2 && ido < bidx))) {
                br2 = r2o;
                bidx = ido;
                bb = bo;
            }
        }
        if (lane == 0 && bb >= 0) {
            const double ds = a.bds[bb];
            const double mref = __dmul_rn(__dmul_rn(a.rho0, ds), ds);
            a.mmax[i] = __dmul_rn(1.05, mref);
            a.mmin[i] = __dmul_rn(0.5, mref);
        }
    }
}

// ------------------------------------------------------------------ split --
__global__ void k_split_flag(int n, const double *m, const double *mmax,
                             uint32_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double mx = mmax[i];
    flag[i] = (mx > 0.0 && m[i] > mx) ? 1u : 0u;
}

__global__ void k_split_collect(int n, const uint32_t *flag,
                                const uint32_t *pos, const int64_t *id,
                                uint64_t *key, uint32_t *val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    key[pos[i]] = (uint64_t)id[i];
    val[pos[i]] = (uint32_t)i;
}

// Parent number r (in id order) writes its six ring children to slots
// n + 6r + k with ids next_id + 6r + k; the centre child stays in place.
__global__ void k_split_emit(SplitArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.count) return;
    const double C[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
    const double S[6] = {0.0, 0.8660254037844386, 0.8660254037844386, 0.0,
                         -0.8660254037844386, -0.8660254037844386};
    const int i = (int)a.parent[r];
    double *f[NSTATE];
    for (int k = 0; k < NSTATE; ++k) f[k] = a.f[k];
    const double m = f[S_M][i], h = f[S_H][i];
    const double mc = __ddiv_rn(m, 7.0);
    const double rad = __dmul_rn(a.eps, h);
    const double hc = __dmul_rn(a.alpha, h);
    for (int k = 0; k < 6; ++k) {
        const int c = a.n + 6 * r + k;
        f[S_X][c] = wrap_rn(a.d, 0, __dadd_rn(f[S_X][i], __dmul_rn(rad, C[k])));
        f[S_Y][c] = wrap_rn(a.d, 1, __dadd_rn(f[S_Y][i], __dmul_rn(rad, S[k])));
        f[S_U][c] = f[S_U][i];
        f[S_V][c] = f[S_V][i];
        f[S_P][c] = f[S_P][i];
        f[S_RHO][c] = f[S_RHO][i];
        f[S_M][c] = mc;
        f[S_H][c] = hc;
        f[S_MMIN][c] = f[S_MMIN][i];
        f[S_MMAX][c] = f[S_MMAX][i];
        if (f[S_DS]) f[S_DS][c] = f[S_DS][i];
        a.id[c] = a.next_id + 6ll * r + k;
    }
    f[S_M][i] = __dsub_rn(m, __dmul_rn(6.0, mc));
    f[S_H][i] = hc;
}

// ------------------------------------------------------------------ merge --
// closest_i: admissible j in N(i) of least (r^2, id_j); admissible: j != i,
// neither to be split, r^2 < ((h_i + h_j)/2)^2, m_i + m_j < max(m_max).
// FP32 bounds for the admissibility test m_i + m_j < max(m_max,i, m_max,j):
// if rd(m_i) + rd(m_j), rounded down, is not below max(ru(m_max)), the FP64
// sum (rounding is monotone and the FP32 bounds are doubles) is not below
// the FP64 maximum either, so the pair is rejected without FP64 work.
__device__ __forceinline__ float2 merge_bounds(double m, double mx, bool alive) {
    if (!alive || !(mx > 0.0) || m > mx) return make_float2(INFINITY, -INFINITY);
    return make_float2(__double2float_rd(m), __double2float_ru(mx));
}

__global__ void k_merge_prep(MergeArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) a.mq[i] = merge_bounds(a.f[S_M][i], a.f[S_MMAX][i], true);
}

template <int T>
__global__ void __launch_bounds__(128) k_merge_closest(MergeArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const double *x = a.f[S_X], *y = a.f[S_Y], *h = a.f[S_H], *m = a.f[S_M],
                 *mmax = a.f[S_MMAX];
    int best = -1;
    double br2 = 0.0;
    long long bid = 0;
    const float2 qi = a.mq[i];
    const bool alive_i = !a.alive_in || a.alive_in[i];
    if (alive_i && qi.y > 0.0f) {
        const double mi = m[i], mxi = mmax[i];
        const double xi = x[i], yi = y[i], hi = h[i];
        const float4 pi = a.pk[i];
        for (uint32_t k = a.off[i] + tm.lane; k < a.off[i + 1]; k += T) {
            const int j = (int)a.list[k];
            if (j == i) continue;
            {   // FP32 mass bound first: it rejects most pairs of a
                // uniform region exactly (see merge_bounds)
                const float2 qj = __ldg(&a.mq[j]);
                if (!(__fadd_rd(qi.x, qj.x) < fmaxf(qi.y, qj.y))) continue;
            }
            {   // FP32 pre-test on the anchor separation (most list
                // entries lie beyond (h_i + h_j)/2): its error is far
                // below the 1e-4 relative margin, so no admissible pair is
                // dropped; the FP64 test below decides
                const float4 pj = __ldg(&a.pk[j]);
                float fx, fy;
                anchor_sep(a.an, pi, pj, fx, fy);
                const float hhf = 0.5f * (pi.z + pj.z);
                if (fmaf(fx, fx, fy * fy) > 1.0001f * hhf * hhf) continue;
            }
            if (a.alive_in && !a.alive_in[j]) continue;
            const double mxj = mmax[j], mj = m[j];
            if (!(mxj > 0.0) || mj > mxj) continue;
            double dx, dy, r2;
            sep_rn(a.d, xi, yi, x[j], y[j], dx, dy, r2);
            const double hh = __dmul_rn(0.5, __dadd_rn(hi, h[j]));
            if (!(r2 < __dmul_rn(hh, hh))) continue;
            const double mx = mxi > mxj ? mxi : mxj;
            if (!(__dadd_rn(mi, mj) < mx)) continue;
            const long long idj = a.id[j];
            if (best < 0 || r2 < br2 || (r2 == br2 && idj < bid)) {
                best = j;
                br2 = r2;
                bid = idj;
            }
        }
    }
    // lexicographic (r^2, id) minimum over the team
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        const int ob = __shfl_xor_sync(tm.mask, best, o);
        const double orr = __shfl_xor_sync(tm.mask, br2, o);
        const long long oid = __shfl_xor_sync(tm.mask, bid, o);
        if (ob >= 0 && (best < 0 || orr < br2 || (orr == br2 && oid < bid))) {
            best = ob;
            br2 = orr;
            bid = oid;
        }
    }
    if (tm.lane == 0) a.closest[i] = best;
}

// Mutually closest pairs merge into the particle with the smaller id
// (Eqs. merged-pos, merged-prop, merged-h with d = 2); alive marks the
// survivors.
__global__ void k_merge_apply(MergeArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (a.alive_in && !a.alive_in[i]) {
        a.alive[i] = 0;
        return;
    }
    const float h0 = a.alive_in ? a.h0[i] : (float)a.f[S_H][i];
    float ds = a.alive_in ? a.dsum[i] : 0.0f;
    const int j = a.closest[i];
    uint32_t alive = 1;
    if (j >= 0 && a.closest[j] == i) {
        if (a.id[i] > a.id[j]) {
            alive = 0;
            a.mq[i] = merge_bounds(0.0, 0.0, false);
        } else {
            double *f[NSTATE];
            for (int k = 0; k < NSTATE; ++k) f[k] = a.f[k];
            const double ma = f[S_M][i], mb = f[S_M][j];
            const double mm = __dadd_rn(ma, mb);
            const double xa = f[S_X][i], ya = f[S_Y][i];
            const double xb = __dadd_rn(xa, min_image(a.d, 0, __dsub_rn(f[S_X][j], xa)));
            const double yb = __dadd_rn(ya, min_image(a.d, 1, __dsub_rn(f[S_Y][j], ya)));
            const double xm = __ddiv_rn(__dadd_rn(__dmul_rn(ma, xa), __dmul_rn(mb, xb)), mm);
            const double ym = __ddiv_rn(__dadd_rn(__dmul_rn(ma, ya), __dmul_rn(mb, yb)), mm);
            const double ax = __dsub_rn(xm, xa), ay = __dsub_rn(ym, ya);
            const double bx = __dsub_rn(xm, xb), by = __dsub_rn(ym, yb);
            const double ra = __dsqrt_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)));
            const double rb = __dsqrt_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)));
            const double den = __dadd_rn(__dmul_rn(ma, W_rn(ra, f[S_H][i])),
                                         __dmul_rn(mb, W_rn(rb, f[S_H][j])));
            const double hm = __dsqrt_rn(__ddiv_rn(__dmul_rn(mm, W_rn(0.0, 1.0)), den));
            auto mw = [&](int k) {
                return __ddiv_rn(__dadd_rn(__dmul_rn(ma, f[k][i]), __dmul_rn(mb, f[k][j])), mm);
            };
            const double un = mw(S_U), vn = mw(S_V), pn = mw(S_P), rn = mw(S_RHO);
            f[S_U][i] = un;
            f[S_V][i] = vn;
            f[S_P][i] = pn;
            f[S_RHO][i] = rn;
            f[S_X][i] = wrap_rn(a.d, 0, xm);
            f[S_Y][i] = wrap_rn(a.d, 1, ym);
            f[S_M][i] = mm;
            f[S_H][i] = hm;
            a.mq[i] = merge_bounds(mm, f[S_MMAX][i], true);
            // reach of the lists for the next round (rounded up)
            ds = __fadd_ru(ds, __double2float_ru(ra));
            if (__fadd_ru(0.5f * __double2float_ru(hm), ds) > a.budget * h0)
                atomicOr(a.stale, 1);
            a.pkw[i] = anchor_record(f[S_X][i], f[S_Y][i], hm, a.lo, a.Ad,
                                     a.invAd, a.an);
        }
    }
    a.h0[i] = h0;
    a.dsum[i] = ds;
    a.alive[i] = alive;
}

// Stream compaction: survivors move to pos[i] in the alternate arrays.
__global__ void k_compact(int n, const uint32_t *alive, const uint32_t *pos,
                          CompactArgs c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !alive[i]) return;
    const uint32_t d = pos[i];
    // a survivor never moves up: pos is the exclusive scan of alive
    if (!SPH_DCHECK(d <= (uint32_t)i)) return;
    for (int k = 0; k < NSTATE; ++k)
        if (c.dst[k]) c.dst[k][d] = c.src[k][i];
    c.idst[d] = c.isrc[i];
}

// ------------------------------------------------------- shift and Taylor --
template <typename R>
struct ShiftIn {
    const R *m, *u, *v, *p;
    __device__ __forceinline__ ShiftIn(const ShiftArgs &a) {
        if (sizeof(R) == sizeof(double)) {
            m = (const R *)a.f[S_M];
            u = (const R *)a.f[S_U];
            v = (const R *)a.f[S_V];
            p = (const R *)a.f[S_P];
        } else {
            m = (const R *)a.mf;
            u = (const R *)a.uf;
            v = (const R *)a.vf;
            p = (const R *)a.pf;
        }
    }
};

// Summation density of every particle (Eq. sd-gather, walls included) and,
// for the h update, the mean fluid-neighbour mass.
template <typename R, int T>
__global__ void __launch_bounds__(128) k_density_mbar(ShiftArgs a, int want_h) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const ShiftIn<R> in(a);
    Sep<R> sp;
    sp.init(a.d, a.f[S_X], a.f[S_Y], a.pk, i);
    const R hi = (R)a.f[S_H][i], hinv = R(1) / hi;
    R rho = 0, msum = 0;
    uint32_t cnt = 0;
    const uint32_t b = a.off[i], e = a.off[i + 1];
    const bool check = want_h && a.filter;
    const float4 pki = check ? a.pk[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const double xi = a.f[S_X][i], yi = a.f[S_Y][i], hid = a.f[S_H][i];
    for (uint32_t k = b + tm.lane; k < e; k += T) {
        const int j = (int)a.list[k];
        R dx, dy, r2;
        sp.get(a.d, a.an, a.f[S_X], a.f[S_Y], a.pk, j, dx, dy, r2);
        // beyond 3 h_i the kernel is exactly zero: for the density alone
        // the entry adds nothing (lists with a skin hold many such
        // entries); the h update's mean mass still counts it
        if (!want_h && !(r2 < R(9) * hi * hi)) continue;
        rho += in.m[j] * qs_w<R>(sqrt(r2) * hinv);   // zero beyond 3 h_i
        if (check) {
            float fx, fy, fr2;
            if (!pred_mixed(a.d, a.an, pki, __ldg(&a.pk[j]), xi, yi, hid,
                            a.f[S_X], a.f[S_Y], a.f[S_H], j, fx, fy, fr2))
                continue;
        }
        msum += in.m[j];
        ++cnt;
    }
    if (a.w.n > 0) {
        for_each_wall<T>(a.w, i, a.d, a.an, a.pk[i], a.f[S_X][i], a.f[S_Y][i], a.f[S_H][i], tm.lane, tm.mask,
                      [&](int k, double, double, double r2) {
            rho += (R)a.w.m[k] * qs_w<R>(sqrt((R)r2) * hinv);
        });
    }
    rho = team_sum<T>(tm.mask, rho);
    msum = team_sum<T>(tm.mask, msum);
    cnt = team_sum<T>(tm.mask, cnt);
    if (tm.lane != 0) return;
    rho *= sigma_norm<R>() * hinv * hinv;
    ((R *)a.rho)[i] = rho;
    if (want_h)
        ((R *)a.hnew)[i] = (R)a.hdx * sqrt((msum / (R)cnt) / rho);
}

// Limited shift (Eqs. shift-deltar, shift-limit; walls included) and the
// Taylor increments grad phi_i . dr_i with grad phi_i = sum_{j != i} V_j
// (phi_j - phi_i) grad_i W(r_ij, h_i) over fluid neighbours.
template <typename R, int T>
__global__ void __launch_bounds__(128) k_shift_compute(ShiftArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const ShiftIn<R> in(a);
    const R *rhoj = (const R *)a.rho;
    Sep<R> sp;
    sp.init(a.d, a.f[S_X], a.f[S_Y], a.pk, i);
    const R hi = (R)a.f[S_H][i], hinv = R(1) / hi;
    const R inv_wxi = R(1) / qs_w<R>(R(XI_INFLECTION));
    const R ui = in.u[i], vi = in.v[i], pi = in.p[i];
    const R rho0 = (R)a.rho0;
    R ax = 0, ay = 0, gux = 0, guy = 0, gvx = 0, gvy = 0, gpx = 0, gpy = 0;
    auto shift = [&](R mj, R hj, R dx, R dy, R r) {
        const R hb = R(0.5) * (hi + hj), hbinv = R(1) / hb;
        R ratio = qs_w<R>(r * hbinv) * inv_wxi;
        ratio *= ratio;
        const R f = (mj / rho0) * (R(1) + R(0.24) * ratio * ratio) *
                    (sigma_norm<R>() * hbinv * hbinv * hbinv) *
                    qs_dw<R>(r * hbinv) / r;
        ax += f * dx;
        ay += f * dy;
    };
    for (uint32_t k = a.off[i] + tm.lane; k < a.off[i + 1]; k += T) {
        const int j = (int)a.list[k];
        if (j == i) continue;
        R dx, dy, r2, hj;
        sp.get(a.d, a.an, a.f[S_X], a.f[S_Y], a.f[S_H], a.pk, j, dx, dy, r2, hj);
        // both kernels vanish beyond 3 max(h_i, h_j): such entries (many in
        // lists with a skin) add exactly nothing
        {
            const R R3 = R(3) * (hi > hj ? hi : hj);
            if (!(r2 < R3 * R3)) continue;
        }
        const R r = sqrt(r2);
        if (!(r > R(0))) continue;
        shift(in.m[j], hj, dx, dy, r);
        const R g = sigma_norm<R>() * hinv * hinv * hinv * qs_dw<R>(r * hinv) / r;
        const R Vg = (in.m[j] / rhoj[j]) * g;
        const R du = in.u[j] - ui, dv = in.v[j] - vi, dp = in.p[j] - pi;
        gux += Vg * du * dx;
        guy += Vg * du * dy;
        gvx += Vg * dv * dx;
        gvy += Vg * dv * dy;
        gpx += Vg * dp * dx;
        gpy += Vg * dp * dy;
    }
    if (a.w.n > 0) {
        for_each_wall<T>(a.w, i, a.d, a.an, a.pk[i], a.f[S_X][i], a.f[S_Y][i], a.f[S_H][i], tm.lane, tm.mask,
                      [&](int k, double dxd, double dyd, double r2) {
            const R r = sqrt((R)r2);
            if (!(r > R(0))) return;
            shift((R)a.w.m[k], (R)a.w.h[k], (R)dxd, (R)dyd, r);
        });
    }
    ax = team_sum<T>(tm.mask, ax);
    ay = team_sum<T>(tm.mask, ay);
    gux = team_sum<T>(tm.mask, gux);
    guy = team_sum<T>(tm.mask, guy);
    gvx = team_sum<T>(tm.mask, gvx);
    gvy = team_sum<T>(tm.mask, gvy);
    gpx = team_sum<T>(tm.mask, gpx);
    gpy = team_sum<T>(tm.mask, gpy);
    if (tm.lane != 0) return;
    const R c = R(-0.5) * hi * hi;
    R sx = c * ax, sy = c * ay;
    const R mag = sqrt(sx * sx + sy * sy), lim = R(0.25) * hi;
    if (mag > lim) {
        const R th = lim / mag;
        sx *= th;
        sy *= th;
    }
    ((R *)a.drx)[i] = sx;
    ((R *)a.dry)[i] = sy;
    ((R *)a.du)[i] = gux * sx + guy * sy;
    ((R *)a.dv)[i] = gvx * sx + gvy * sy;
    ((R *)a.dp)[i] = gpx * sx + gpy * sy;
}

template <typename R>
__global__ void k_shift_apply(ShiftArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.f[S_X][i] = wrap_rn(a.d, 0, a.f[S_X][i] + (double)((const R *)a.drx)[i]);
    a.f[S_Y][i] = wrap_rn(a.d, 1, a.f[S_Y][i] + (double)((const R *)a.dry)[i]);
    a.f[S_U][i] += (double)((const R *)a.du)[i];
    a.f[S_V][i] += (double)((const R *)a.dv)[i];
    a.f[S_P][i] += (double)((const R *)a.dp)[i];
    a.f[S_RHO][i] = (double)((const R *)a.rho)[i];
}

template <typename R>
__global__ void k_h_apply(ShiftArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    a.f[S_H][i] = (double)((const R *)a.hnew)[i];
    a.f[S_RHO][i] = (double)((const R *)a.rho)[i];
}

// Deterministic two-stage sum of the masses.
__global__ void k_mass_partial(int n, const double *m, double *part) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256)
        acc += m[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_mass_final(int nb, const double *part, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[b];
        *out = acc;
    }
}

// ------------------------------------------------------------- launchers --
static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

void launch_bg_mref(cudaStream_t s, const BgArgs &a) {
    if (a.n <= 0) return;
    cudaMemsetAsync(a.nqueue, 0, sizeof(uint32_t), s);
    with_team(a.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_bg_mref<T><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
    });
    k_bg_nearest<<<152, 256, 0, s>>>(a);
}
void launch_split_flag(cudaStream_t s, int n, const double *m,
                       const double *mmax, uint32_t *flag) {
    if (n > 0) k_split_flag<<<nblk(n, 256), 256, 0, s>>>(n, m, mmax, flag);
}
void launch_split_collect(cudaStream_t s, int n, const uint32_t *flag,
                          const uint32_t *pos, const int64_t *id,
                          uint64_t *key, uint32_t *val) {
    if (n > 0)
        k_split_collect<<<nblk(n, 256), 256, 0, s>>>(n, flag, pos, id, key, val);
}
void launch_split_emit(cudaStream_t s, const SplitArgs &a) {
    if (a.count > 0) k_split_emit<<<nblk(a.count, 128), 128, 0, s>>>(a);
}
void launch_merge(cudaStream_t s, const MergeArgs &a) {
    if (a.n <= 0) return;
    if (!a.alive_in) k_merge_prep<<<nblk(a.n, 256), 256, 0, s>>>(a);
    with_team(a.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_merge_closest<T><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
    });
    k_merge_apply<<<nblk(a.n, 128), 128, 0, s>>>(a);
}
void launch_compact(cudaStream_t s, int n, const uint32_t *alive,
                    const uint32_t *pos, const CompactArgs &c) {
    if (n > 0) k_compact<<<nblk(n, 256), 256, 0, s>>>(n, alive, pos, c);
}
template <typename R, int T>
static void shift_round_T(cudaStream_t s, const ShiftArgs &a) {
    k_density_mbar<R, T><<<nblk(a.n * T, 128), 128, 0, s>>>(a, 0);
    k_shift_compute<R, T><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
    k_shift_apply<R><<<nblk(a.n, 256), 256, 0, s>>>(a);
}
template <typename R>
static void shift_round_R(cudaStream_t s, const ShiftArgs &a) {
    with_team(a.n, [&](auto t) { shift_round_T<R, decltype(t)::value>(s, a); });
}
void launch_shift_round(cudaStream_t s, const ShiftArgs &a, bool mixed) {
    if (a.n <= 0) return;
    if (mixed)
        shift_round_R<float>(s, a);
    else
        shift_round_R<double>(s, a);
}
template <typename R, int T>
static void h_update_T(cudaStream_t s, const ShiftArgs &a) {
    k_density_mbar<R, T><<<nblk(a.n * T, 128), 128, 0, s>>>(a, 1);
    k_h_apply<R><<<nblk(a.n, 256), 256, 0, s>>>(a);
}
template <typename R>
static void h_update_R(cudaStream_t s, const ShiftArgs &a) {
    with_team(a.n, [&](auto t) { h_update_T<R, decltype(t)::value>(s, a); });
}
void launch_h_update(cudaStream_t s, const ShiftArgs &a, bool mixed) {
    if (a.n <= 0) return;
    if (mixed)
        h_update_R<float>(s, a);
    else
        h_update_R<double>(s, a);
}
int launch_mass_sum(cudaStream_t s, int n, const double *m, double *part,
                    double *out) {
    int nb = std::max(1, std::min(nblk(n, 256), 256));
    if (nb == 1) {   // small sets: the block's sum is the total
        k_mass_partial<<<1, 256, 0, s>>>(n, m, out);
        return 1;
    }
    k_mass_partial<<<nb, 256, 0, s>>>(n, m, part);
    k_mass_final<<<1, 32, 0, s>>>(nb, part, out);
    return 2;
}

SPH_DEBUG_COUNTER(debug_failures_adapt)

}  // namespace sph
