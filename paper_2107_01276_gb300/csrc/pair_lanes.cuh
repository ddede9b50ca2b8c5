// Per-particle arithmetic of the two gather passes of one right-hand side
// (section 2): the accumulators of particle i, the contribution of one
// neighbour j, the final per-particle formulas, and the loops over a range
// of list entries.  The single-instance and batched pass kernels
// (pair_passes.cu) share them, so an instance's pairs are evaluated with the
// same operations in the same order however it is launched.
#pragma once

#include "debug_checks.cuh"
#include "kernels.cuh"
#include "pair_passes.cuh"
#include "team.cuh"

namespace sph {

// List entries whose neighbour records a mixed-path pass loads ahead.
#ifndef SPH_UNROLL_A
#define SPH_UNROLL_A 4
#endif
#ifndef SPH_UNROLL_B
#define SPH_UNROLL_B 2
#endif
constexpr int UNROLL_A = SPH_UNROLL_A;
constexpr int UNROLL_B = SPH_UNROLL_B;

// Membership test of a list entry when the lists carry a skin: the exact
// predicate of N(i) on the separation the pass already has (FP32 band test
// with the FP64 predicate inside the band on the mixed path; the FP64
// predicate on the FP64 path).
template <typename R>
__device__ __forceinline__ bool skin_member(const Domain &d, const Anchor &an,
                                            R r2, R hi, R hj, double xi,
                                            double yi, double hid,
                                            const double *x, const double *y,
                                            const double *h, int j) {
    if constexpr (sizeof(R) == 4) {
        return member_r2(d, an, r2, hi, hj, xi, yi, hid, x, y, h, j);
    } else {
        return pred_fp64(d, xi, yi, hid, __ldg(&x[j]), __ldg(&y[j]), __ldg(&h[j]));
    }
}

// ---------------------------------------------------------------- pass A --
// Summation density (Eq. sd-gather), beta (Eq. beta), p_avg (Eq. pavg, N_i
// counts i), shift dr (Eq. shift-deltar, volume m_j / rho0, W ratio
// against the kernel at its inflection point for h_ij = (h_i + h_j)/2),
// limited to 0.25 h_i (Eq. shift-limit).  finish() also writes the two
// per-particle records pass B gathers: {m, V = m/rho, rho, 1/(rho^2 beta)}
// and {p, u, v, 1/h}.
template <typename R>
struct PassALane {
    R hi, hinv, inv_wxi;
    R rho, srw, psum, ax, ay;
    int cnt;

    __device__ __forceinline__ void init(const PassAArgs<R> &a, int i) {
        hi = (R)a.h[i];
        hinv = R(1) / hi;
        inv_wxi = R(1) / qs_w<R>(R(XI_INFLECTION));
        rho = srw = psum = ax = ay = R(0);
        cnt = 0;
    }

    // member j (self: j == i) at separation r_i - r_j = (dx, dy), r2 = r^2
    __device__ __forceinline__ void pair(R mj, R hj, R pj, bool self, R dx,
                                         R dy, R r2) {
        const R rinv = r2 > R(0) ? frsqrt(r2) : R(0);
        const R r = r2 * rinv;
        const R q = r * hinv;
        rho += mj * qs_w<R>(q);
        srw += mj * r * qs_dw<R>(q);
        psum += pj;
        cnt += 1;
        if (!self && r > R(0)) {
            const R hbinv = fdiv(R(2), hi + hj);
            const R qb = r * hbinv;
            R ratio = qs_w<R>(qb) * inv_wxi;
            ratio *= ratio;
            const R f = mj * (R(1) + R(0.24) * ratio * ratio) *
                        (sigma_norm<R>() * hbinv * hbinv * hbinv) *
                        qs_dw<R>(qb) * rinv;
            ax += f * dx;
            ay += f * dy;
        }
    }

    // wall neighbours of particle i (section 2.2): mass m_w in rho, beta
    // and the shift, p_w in p_avg
    template <int T>
    __device__ __forceinline__ void walls(const PassAArgs<R> &a, int i,
                                          const Team<T> &tm) {
        if (a.w.n <= 0) return;
        for_each_wall<T>(a.w, i, a.d, a.an, a.pk[i], a.x[i], a.y[i], a.h[i],
                         tm.lane, tm.mask,
                         [&](int k, double dxd, double dyd, double r2d) {
            pair((R)a.w.m[k], (R)a.w.h[k], (R)a.w.p[k], false, (R)dxd,
                 (R)dyd, (R)r2d);
        });
    }

    template <int T>
    __device__ __forceinline__ void finish(const PassAArgs<R> &a, int i,
                                           const Team<T> &tm) {
        rho = team_sum<T>(tm.mask, rho);
        srw = team_sum<T>(tm.mask, srw);
        psum = team_sum<T>(tm.mask, psum);
        ax = team_sum<T>(tm.mask, ax);
        ay = team_sum<T>(tm.mask, ay);
        cnt = team_sum<T>(tm.mask, cnt);
        if (tm.lane != 0) return;
        const R sig = sigma_norm<R>() * hinv * hinv;
        rho *= sig;
        const R beta = -(sig * hinv * srw) / (rho * R(2));
        R drx = R(0), dry = R(0);
        if (beta != R(0)) {
            const R c = R(-0.5) * hi * hi / (R)a.rho0;
            drx = c * ax;
            dry = c * ay;
        }
        const R mag = sqrt(drx * drx + dry * dry);
        const R lim = R(0.25) * hi;
        if (mag > lim) {
            const R th = lim / mag;
            drx *= th;
            dry *= th;
        }
        const R mi = a.m[i];
        const R V = mi / rho;
        const R rb2 = beta != R(0) ? R(1) / (rho * rho * beta) : R(0);
        a.rho[i] = rho;
        a.beta[i] = beta;
        a.pavg[i] = psum / (R)cnt;
        a.nnb[i] = cnt;
        a.drx[i] = drx;
        a.dry[i] = dry;
        a.V[i] = V;
        a.rb2[i] = rb2;
        typename V4<R>::T A, B;
        A.x = mi; A.y = V; A.z = rho; A.w = rb2;
        B.x = a.p[i]; B.y = a.u[i]; B.z = a.v[i]; B.w = hinv;
        a.nbA[i] = A;
        a.nbB[i] = B;
    }
};

// ---------------------------------------------------------------- pass B --
// EDAC pressure rate (Eq. edac:sph) and momentum rate (Eq. mom-sph without
// the A_i/A_j stresses and third line, unused per the paper's remark):
//   dp/dt = rho0 c^2/beta_i sum V_j u_ij.gW_i
//         + 1/beta_i sum V_j nu_ij (p_i - p_j) r_ij.gW_ij / (r^2 + eta)
//         + rho_i sum m_j (dr_i/dt).(P_i gW_i + P_j gW_j)
//   du/dt = -sum m_j (P_i gW_i + P_j gW_j)
//         + 1/beta_i sum m_j 4 nu/(rho_i + rho_j) r_ij.gW_ij/(r^2 + eta) u_ij
// gW_i = grad W(r_ij, h_i), gW_ij the mean of gW_i and gW_j (Eq. dw-avg),
// nu_ij the Cleary mean 4 nu_i nu_j/(nu_i + nu_j) of nu_e = alpha_e c h / 8
// (Eqs. edac-alpha, nu-cleary), which equals (alpha_e c / 2) / (1/h_i +
// 1/h_j); eta = 0.001 h_i^2, P_j = (p_j - p_avg,i) / (rho_j^2 beta_j).
// Wall neighbours (section 2.2): prescribed wall velocity in the divergence
// sum, extrapolated velocity in the viscous sum, rho_w = rho0, beta_w = 1.
// Every term carries grad W(r, h_i) or grad W(r, h_j), so a pair with
// r >= 3 max(h_i, h_j) -- or r = 0, i itself -- adds exactly zero.
// Factors common to all pairs of i are applied once, in finish(): the
// Cleary numerator alpha_e c / 2 of the diffusion sum, the 4 nu of the
// viscous sum, and the transport sum, which is (dr_i/dt) . sum m_j (P_i
// gW_i + P_j gW_j) = -(dr_i/dt) . (pressure force sum).
template <typename R>
struct PassBLane {
    R hinv, dsig_i, rho_i, pi, ui, vi, pavg_i, Pi, eta;
    bool dden_on;
    R div, diff, fax, fay, vx, vy;

    // false: beta_i = 0 (no neighbour at r > 0), zero rates (reading R1)
    __device__ __forceinline__ bool init(const PassBArgs<R> &a, int i) {
        const R rb2i = a.rb2[i];
        const R beta_i = a.beta[i];
        div = diff = fax = fay = vx = vy = R(0);
        if (beta_i == R(0)) return false;
        const typename V4<R>::T Bi = a.nbB[i];
        hinv = Bi.w;
        dsig_i = sigma_norm<R>() * hinv * hinv * hinv;
        rho_i = a.rho[i];
        pi = Bi.x;
        ui = Bi.y;
        vi = Bi.z;
        pavg_i = a.pavg[i];
        Pi = (pi - pavg_i) * rb2i;
        const R hi = R(1) / hinv;
        eta = R(0.001) * hi * hi;
        dden_on = a.diff_denominator != 0;
        return true;
    }

    // one neighbour's contributions; (ujx, ujy): velocity in the divergence
    // sum, (ugx, ugy): velocity in the viscous sum
    __device__ __forceinline__ void pair(R dx, R dy, R r2, R hjinv, R mj,
                                         R Vj, R rho_j, R Pj, R pj, R ujx,
                                         R ujy, R ugx, R ugy) {
        R gi = 0, gj = 0;
        if (r2 > R(0)) {
            const R rinv = frsqrt(r2);
            const R r = r2 * rinv;
            gi = dsig_i * qs_dw<R>(r * hinv) * rinv;
            gj = sigma_norm<R>() * hjinv * hjinv * hjinv *
                 qs_dw<R>(r * hjinv) * rinv;
        }
        const R rdg = R(0.5) * (gi + gj) * r2;
        // nu_ij / (alpha_e c / 2)
        const R nu_ij = fdiv(R(1), hinv + hjinv);
        const R inv_reta = fdiv(R(1), r2 + eta);
        const R uij = ui - ujx, vij = vi - ujy;
        div += Vj * gi * (uij * dx + vij * dy);
        diff += Vj * nu_ij * (pi - pj) * rdg * (dden_on ? inv_reta : R(1));
        const R mfp = mj * (Pi * gi + Pj * gj);
        fax -= mfp * dx;
        fay -= mfp * dy;
        // m_j 4 nu/(rho_i + rho_j) r.gW_ij/(r^2 + eta) / (4 nu)
        const R visc = fdiv(mj * rdg * inv_reta, rho_i + rho_j);
        vx += visc * (ui - ugx);
        vy += visc * (vi - ugy);
    }

    // list neighbour j with its pass-B records A = {m, V, rho, 1/(rho^2
    // beta)}, B = {p, u, v, 1/h}; pref: p_avg,i, or p_avg,j (literal
    // reading, pavg_mode 1)
    template <typename V>
    __device__ __forceinline__ void pair_rec(R dx, R dy, R r2, const V &A,
                                             const V &B, R pref) {
        pair(dx, dy, r2, B.w, A.x, A.y, A.z, (B.x - pref) * A.w, B.x, B.y,
             B.z, B.y, B.z);
    }

    template <int T>
    __device__ __forceinline__ void walls(const PassBArgs<R> &a, int i,
                                          const Team<T> &tm) {
        if (a.w.n <= 0) return;
        const R rho0 = (R)a.rho0;
        const bool literal = a.pavg_mode != 0;
        for_each_wall<T>(a.w, i, a.d, a.an, a.pk[i], a.x[i], a.y[i], a.h[i],
                         tm.lane, tm.mask,
                         [&](int k, double dxd, double dyd, double r2d) {
            const R mk = (R)a.w.m[k], pk = (R)a.w.p[k];
            const R pref = literal ? R(0) : pavg_i;
            pair((R)dxd, (R)dyd, (R)r2d, R(1) / (R)a.w.h[k], mk, mk / rho0,
                 rho0, (pk - pref) / (rho0 * rho0), pk, (R)a.w.uw[k],
                 (R)a.w.vw[k], (R)a.w.ugx[k], (R)a.w.ugy[k]);
        });
    }

    // on: init() returned true (else the rates are zero)
    template <int T>
    __device__ __forceinline__ void finish(const PassBArgs<R> &a, int i,
                                           const Team<T> &tm, bool on) {
        div = team_sum<T>(tm.mask, div);
        diff = team_sum<T>(tm.mask, diff);
        fax = team_sum<T>(tm.mask, fax);
        fay = team_sum<T>(tm.mask, fay);
        vx = team_sum<T>(tm.mask, vx);
        vy = team_sum<T>(tm.mask, vy);
        if (tm.lane != 0) return;
        if (!on) {
            a.dpdt[i] = R(0);
            a.dudt[i] = R(0);
            a.dvdt[i] = R(0);
            return;
        }
        const R beta_i = a.beta[i];
        const R rf = a.rho_factor ? rho_i : R(1);
        // (u~ - u) = dr / dt by the reciprocal the time-step kernel stores
        const R idt = (R)a.dt[1];
        const R tvf = -(a.drx[i] * idt * fax + a.dry[i] * idt * fay);
        const R half_ac = R(0.5) * (R)a.alpha_e * (R)a.cs;
        const R four_nu = R(4) * (R)a.nu;
        const R dpdt = ((R)a.rho0 * (R)a.cs * (R)a.cs / beta_i) * div +
                       half_ac * diff / beta_i + rf * tvf;
        const R dudt = fax + four_nu * vx / beta_i;
        const R dvdt = fay + four_nu * vy / beta_i;
        a.dpdt[i] = dpdt;
        a.dudt[i] = dudt;
        a.dvdt[i] = dvdt;
        if (!isfinite((double)dpdt) || !isfinite((double)dudt) ||
            !isfinite((double)dvdt))
            atomicOr(a.nonfinite, 1);
    }
};

// Pass A over the list entries [b, e) of particle i, in list order (team
// lane t takes entries b + t, b + t + T, ...).
template <typename R, int T>
__device__ __forceinline__ void pass_a_list(const PassAArgs<R> &a, int i,
                                            PassALane<R> &L, const Team<T> &tm,
                                            uint32_t b, uint32_t e) {
    Sep<R> sp;
    sp.init(a.d, a.x, a.y, a.pk, i);
    const R hi = L.hi;
    const double xid = a.x[i], yid = a.y[i], hid = a.h[i];
    if constexpr (sizeof(R) == 4) {
        // U list entries per step, their records loaded before any is used
        // (more loads in flight per warp)
        auto body = [&](int j, const float4 &pj, R mj, R pjv) {
            R dx, dy;
            anchor_sep(a.an, sp.pi, pj, dx, dy);
            const R r2 = fmaf(dx, dx, dy * dy);
            if (a.filter && !skin_member<R>(a.d, a.an, r2, hi, pj.z, xid, yid,
                                            hid, a.x, a.y, a.h, j))
                return;
            L.pair(mj, pj.z, pjv, j == i, dx, dy, r2);
        };
        constexpr int U = UNROLL_A;
        uint32_t k = b + tm.lane;
        for (; k + (U - 1) * T < e; k += U * T) {
            int jj[U];
            float4 pp[U];
            R mm[U], qq[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                jj[u] = (int)__ldg(&a.list[k + u * T]);
                // an index out of range (debug builds) reads i instead
                if (!SPH_DCHECK((unsigned)jj[u] < (unsigned)a.n)) jj[u] = i;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                pp[u] = __ldg(&a.pk[jj[u]]);
                mm[u] = a.m[jj[u]];
                qq[u] = a.p[jj[u]];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) body(jj[u], pp[u], mm[u], qq[u]);
        }
        for (; k < e; k += T) {
            int j = (int)__ldg(&a.list[k]);
            if (!SPH_DCHECK((unsigned)j < (unsigned)a.n)) j = i;
            body(j, __ldg(&a.pk[j]), a.m[j], a.p[j]);
        }
    } else {
        for (uint32_t k = b + tm.lane; k < e; k += T) {
            const int j = (int)__ldg(&a.list[k]);
            if (!SPH_DCHECK((unsigned)j < (unsigned)a.n)) continue;
            R dx, dy, r2, hj;
            sp.get(a.d, a.an, a.x, a.y, a.h, a.pk, j, dx, dy, r2, hj);
            if (a.filter && !skin_member<R>(a.d, a.an, r2, hi, hj, xid, yid, hid,
                                            a.x, a.y, a.h, j))
                continue;
            L.pair(a.m[j], hj, a.p[j], j == i, dx, dy, r2);
        }
    }
}

// Pass B over the list entries [b, e) of particle i, in list order.
template <typename R, int T>
__device__ __forceinline__ void pass_b_list(const PassBArgs<R> &a, int i,
                                            PassBLane<R> &L, const Team<T> &tm,
                                            uint32_t b, uint32_t e) {
    Sep<R> sp;
    sp.init(a.d, a.x, a.y, a.pk, i);
    const R pavg_i = L.pavg_i;
    const bool literal = a.pavg_mode != 0;
    const double xid = a.x[i], yid = a.y[i], hid = a.h[i];
    const R hpk = (R)a.pk[i].z;   // h_i as the list builder saw it
    if constexpr (sizeof(R) == 4) {
        // neither a membership test for skin entries nor a test for i
        // itself: both add exactly zero
        auto body = [&](int j, const float4 &pj, const float4 &A,
                        const float4 &B) {
            R dx, dy;
            anchor_sep(a.an, sp.pi, pj, dx, dy);
            L.pair_rec(dx, dy, fmaf(dx, dx, dy * dy), A, B,
                       literal ? a.pavg[j] : pavg_i);
        };
        constexpr int U = UNROLL_B;
        uint32_t k = b + tm.lane;
        for (; k + (U - 1) * T < e; k += U * T) {
            int jj[U];
            float4 pp[U], AA[U], BB[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                jj[u] = (int)__ldg(&a.list[k + u * T]);
                if (!SPH_DCHECK((unsigned)jj[u] < (unsigned)a.n)) jj[u] = i;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                pp[u] = __ldg(&a.pk[jj[u]]);
                AA[u] = a.nbA[jj[u]];
                BB[u] = a.nbB[jj[u]];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) body(jj[u], pp[u], AA[u], BB[u]);
        }
        for (; k < e; k += T) {
            int j = (int)__ldg(&a.list[k]);
            if (!SPH_DCHECK((unsigned)j < (unsigned)a.n)) j = i;
            body(j, __ldg(&a.pk[j]), a.nbA[j], a.nbB[j]);
        }
    } else {
        for (uint32_t k = b + tm.lane; k < e; k += T) {
            const int j = (int)__ldg(&a.list[k]);
            if (!SPH_DCHECK((unsigned)j < (unsigned)a.n)) continue;
            if (j == i) continue;
            R dx, dy, r2;
            if (a.filter) {
                R hj;
                sp.get(a.d, a.an, a.x, a.y, a.h, a.pk, j, dx, dy, r2, hj);
                if (!skin_member<R>(a.d, a.an, r2, hpk, hj, xid, yid, hid, a.x,
                                    a.y, a.h, j))
                    continue;
            } else {
                sp.get(a.d, a.an, a.x, a.y, a.pk, j, dx, dy, r2);
            }
            L.pair_rec(dx, dy, r2, a.nbA[j], a.nbB[j], literal ? a.pavg[j] : pavg_i);
        }
    }
}

}  // namespace sph
