// Gather pair loops of one right-hand-side evaluation (section 2), the PEC
// stages (section 2.4) and the time-step reduction (Eq. timestep).
//
// Thread per particle over the key-sorted order: neighbouring lanes sit in
// the same or adjacent cells, so a warp's candidate loads hit the same
// lines.  Templated on the pair-arithmetic type R (double: FP64 path,
// float: mixed path); positions and the neighbour predicate stay FP64.
#include <float.h>

#include <algorithm>

#include "batch.cuh"
#include "kernels.cuh"
#include "lists.cuh"
#include "neighbors.cuh"
#include "pair_lanes.cuh"
#include "pair_passes.cuh"
#include "team.cuh"

namespace sph {

// resident 128-thread blocks per SM the mixed passes are compiled for
#ifndef SPH_PASS_A_BLOCKS
#define SPH_PASS_A_BLOCKS 8
#endif
#ifndef SPH_PASS_B_BLOCKS
#define SPH_PASS_B_BLOCKS 8
#endif
constexpr int PASS_A_BLOCKS = SPH_PASS_A_BLOCKS;
constexpr int PASS_B_BLOCKS = SPH_PASS_B_BLOCKS;
// Team forms (T > 1: small and walled sets) and the batched forms keep six
// and five blocks (80 / 96 registers): at the eight-block cap their wall
// loops spill.
template <typename R, int T>
constexpr int pass_blocks(int lane1) {
    return sizeof(R) == 4 ? (T == 1 ? lane1 : 6) : 1;
}

// ---------------------------------------------------------------- pass A --
// Pass A of particle i over its list (arithmetic in PassALane): a team of T
// threads shares particle i.  WALLS = false: a set without wall particles,
// compiled without the wall loop (whose registers made the one-lane pass B
// spill at the eight-block bound).
template <typename R, int T, bool WALLS = true>
__device__ __forceinline__ void pass_a_at(const PassAArgs<R> &a, int i,
                                          const Team<T> &tm) {
    PassALane<R> L;
    L.init(a, i);
    pass_a_list<R, T>(a, i, L, tm, a.off[i], a.off[i + 1]);
    if constexpr (WALLS) L.walls(a, i, tm);
    L.finish(a, i, tm);
}

template <typename R, int T, bool WALLS>
__global__ void __launch_bounds__(128, (pass_blocks<R, T>(PASS_A_BLOCKS)))
    k_pass_a(PassAArgs<R> a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    pass_a_at<R, T, WALLS>(a, i, tm);
}

// ---------------------------------------------------------------- pass B --
// Pass B of particle i over its list (arithmetic in PassBLane).
// (float, one lane per particle: at most 64 registers, eight 128-thread
// blocks per SM, measured faster than six at 80 registers on the graded
// 1:250 strip)
template <typename R, int T, bool WALLS = true>
__device__ __forceinline__ void pass_b_at(const PassBArgs<R> &a, int i,
                                          const Team<T> &tm) {
    PassBLane<R> L;
    if (!L.init(a, i)) {
        if (tm.lane == 0) {
            a.dpdt[i] = R(0);
            a.dudt[i] = R(0);
            a.dvdt[i] = R(0);
        }
        return;
    }
    pass_b_list<R, T>(a, i, L, tm, a.off[i], a.off[i + 1]);
    if constexpr (WALLS) L.walls(a, i, tm);
    L.finish(a, i, tm, true);
}

template <typename R, int T, bool WALLS>
__global__ void __launch_bounds__(128, (pass_blocks<R, T>(PASS_B_BLOCKS)))
    k_pass_b(PassBArgs<R> a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    pass_b_at<R, T, WALLS>(a, i, tm);
}

// --------------------------------------------------------- wall BC -----
// Section 2.2 (Adami dummy walls), per wall particle w over fluid f with
// W_wf = W(r_wf, (h_w + h_f)/2): u^ = sum u_f W / sum W (Eq. shepard),
// u_ghost = 2 u_wall - u^ (Eq. bc-wall), p_w = sum p_f W / sum W (Eq.
// bc-pre with g = a_w = 0); p_w = 0 and u^ = 0 without fluid in range.
template <int T>
__device__ __forceinline__ void wall_bc_at(const WallBcArgs &a, int k,
                                           const Team<T> &tm) {
    const double xw = a.w.x[k], yw = a.w.y[k], hw = a.w.h[k];
    const float4 pw = a.w.pk[k];
    const float2 q = anchor_rel(a.an, pw);
    double sw = 0, su = 0, sv = 0, sp = 0;
    for_each_candidate_team<T>(a.g, a.d, 0, q.x, q.y, pw.z, a.qscale, tm.lane,
                               tm.mask, [](uint32_t, uint32_t) { return true; },
                               [&](uint32_t f) {
        {
            float fx, fy, fr2;
            if (!pred_mixed(a.d, a.an, pw, __ldg(&a.pk[f]), xw, yw, hw, a.x,
                            a.y, a.h, (int)f, fx, fy, fr2))
                return;
            const double xf = __ldg(&a.x[f]), yf = __ldg(&a.y[f]),
                         hf = __ldg(&a.h[f]);
            const double dx = min_image(a.d, 0, xw - xf);
            const double dy = min_image(a.d, 1, yw - yf);
            const double hbinv = 1.0 / (0.5 * (hw + hf));
            const double W = sigma_norm<double>() * hbinv * hbinv *
                             qs_w<double>(sqrt(dx * dx + dy * dy) * hbinv);
            sw += W;
            su += a.u[f] * W;
            sv += a.v[f] * W;
            sp += a.p[f] * W;
        }
    });
    sw = team_sum<T>(tm.mask, sw);
    su = team_sum<T>(tm.mask, su);
    sv = team_sum<T>(tm.mask, sv);
    sp = team_sum<T>(tm.mask, sp);
    if (tm.lane != 0) return;
    double uh = 0, vh = 0, p = 0;
    if (sw > 0) {
        uh = su / sw;
        vh = sv / sw;
        p = sp / sw;
    }
    a.pw[k] = p;
    a.ugx[k] = 2.0 * a.w.uw[k] - uh;
    a.ugy[k] = 2.0 * a.w.vw[k] - vh;
}

template <int T>
__global__ void __launch_bounds__(128) k_wall_bc(WallBcArgs a) {
    const Team<T> tm;
    const int k = Team<T>::particle();
    if (k >= a.w.n) return;
    wall_bc_at<T>(a, k, tm);
}

// ------------------------------------------------------------ wall lists --
template <int T>
__global__ void __launch_bounds__(128) k_wall_lists(WallListArgs a, int fill) {
    const Team<T> tm;
    const int k = Team<T>::particle();
    if (k >= a.w.n) return;
    const float4 pw = a.w.pk[k];
    const float2 q = anchor_rel(a.an, pw);
    for_each_candidate_team<T>(a.g, a.d, 0, q.x, q.y, pw.z, a.reach, tm.lane,
                               tm.mask, [](uint32_t, uint32_t) { return true; },
                               [&](uint32_t j) {
        const float4 pj = __ldg(&a.pk[j]);
        float dx, dy;
        anchor_sep(a.an, pw, pj, dx, dy);
        const float R = a.reach * 3.0f * fmaxf(pw.z, pj.z);
        if (!(fmaf(dx, dx, dy * dy) < R * R)) return;
        if (!fill) {
            atomicAdd(&a.cnt[j], 1u);
        } else {
            const uint32_t p = a.off[j] + atomicAdd(&a.cur[j], 1u);
            if (p < a.cap)
                a.list[p] = (uint32_t)k;
            else
                atomicOr(a.overflow, 1);
        }
    });
}

// ---------------------------------------------------------- force on solid --
// Section "Force computation", Eq. force-sph, for wall particle k over its
// fluid neighbours j; FP64 sums (a team of T lanes per wall particle).
template <typename R, int T>
__global__ void __launch_bounds__(128) k_forces(ForceArgs<R> a) {
    const Team<T> tm;
    const int k = Team<T>::particle();
    if (k >= a.w.n) return;
    const double xw = a.w.x[k], yw = a.w.y[k], hw = a.w.h[k];
    const float4 pw = a.w.pk[k];
    const float2 q = anchor_rel(a.an, pw);
    const double Pw = a.w.p[k] / (a.rho0 * a.rho0);
    const double ugx = a.w.ugx[k], ugy = a.w.ugy[k];
    const double eta = 0.001 * hw * hw;
    const double sw = sigma_norm<double>() / (hw * hw * hw);
    double fpx = 0, fpy = 0, fvx = 0, fvy = 0;
    for_each_candidate_team<T>(a.g, a.d, 0, q.x, q.y, pw.z, 1.0f, tm.lane,
                               tm.mask, [](uint32_t, uint32_t) { return true; },
                               [&](uint32_t j) {
        float fx, fy, fr2;
        if (!pred_mixed(a.d, a.an, pw, __ldg(&a.pk[j]), xw, yw, hw, a.x, a.y,
                        a.h, (int)j, fx, fy, fr2))
            return;
        const double beta_j = (double)a.beta[j];
        if (beta_j == 0.0) return;
        const double dx = min_image(a.d, 0, xw - a.x[j]);
        const double dy = min_image(a.d, 1, yw - a.y[j]);
        const double r2 = dx * dx + dy * dy;
        double gw = 0.0, gj = 0.0;
        if (r2 > 0.0) {
            const double r = sqrt(r2), hj = a.h[j];
            gw = sw * qs_dw<double>(r / hw) / r;
            gj = sigma_norm<double>() / (hj * hj * hj) * qs_dw<double>(r / hj) / r;
        }
        const double rho_j = (double)a.rho[j], mj = a.m[j];
        const double Pj = a.p[j] / (rho_j * rho_j * beta_j);
        const double fp = mj * (Pw * gw + Pj * gj);
        fpx -= fp * dx;
        fpy -= fp * dy;
        const double visc = mj * (4.0 * a.nu / (a.rho0 + rho_j)) *
                            (0.5 * (gw + gj) * r2) / (r2 + eta);
        fvx += visc * (ugx - a.u[j]);
        fvy += visc * (ugy - a.v[j]);
    });
    fpx = team_sum<T>(tm.mask, fpx);
    fpy = team_sum<T>(tm.mask, fpy);
    fvx = team_sum<T>(tm.mask, fvx);
    fvy = team_sum<T>(tm.mask, fvy);
    if (tm.lane != 0) return;
    const double mw = a.w.m[k];   // beta_w = 1
    a.fw[4 * k] = mw * fpx;
    a.fw[4 * k + 1] = mw * fpy;
    a.fw[4 * k + 2] = mw * fvx;
    a.fw[4 * k + 3] = mw * fvy;
}

// One block: fixed-order sums of the four components (each thread a
// strided share, then a tree over the threads) and the load-order copy.
__global__ void __launch_bounds__(256)
    k_forces_total(int nw, const double *fw, const int64_t *id, double *out,
                   double *total) {
    __shared__ double s[4][256];
    double acc[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < nw; k += 256) {
        const int64_t o = id[k];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[c] += fw[4 * k + c];
            out[4 * o + c] = fw[4 * k + c];
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 4) total[threadIdx.x] = s[threadIdx.x][0];
}

// ---------------------------------------------------- neighbour CSR dump --
__global__ void k_nbr_ids(int n, const uint32_t *off, const uint32_t *list,
                          const int64_t *id, int64_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (uint32_t k = off[i]; k < off[i + 1]; ++k) out[k] = id[list[k]];
}

// ------------------------------------------------------------ PEC stages --
// Section 2.4: u' = u0 + f dt du/dt; u~' = u' + dr/dt; r' = r0 + f dt u~';
// p' = p0 + f dt dp/dt, with f = 1/2 (predict) or 1 (correct); FP64,
// explicitly rounded; periodic axes wrapped back into the box; then, with
// a sponge layer, the corrector relaxes u, v, p towards (U, 0, 0) in it.
template <typename R>
__device__ __forceinline__ void pec_at(const PecArgs<R> &a, int i) {
    const double dt = a.dt[0], idt = a.dt[1];
    const double fdt = __dmul_rn(a.f, dt);
    double x0, y0, u0, v0, p0;
    if (a.save) {
        x0 = a.x[i];
        y0 = a.y[i];
        u0 = a.u[i];
        v0 = a.v[i];
        p0 = a.p[i];
        ((double *)a.x0)[i] = x0;
        ((double *)a.y0)[i] = y0;
        ((double *)a.u0)[i] = u0;
        ((double *)a.v0)[i] = v0;
        ((double *)a.p0)[i] = p0;
    } else {
        x0 = a.x0[i];
        y0 = a.y0[i];
        u0 = a.u0[i];
        v0 = a.v0[i];
        p0 = a.p0[i];
    }
    const double un = __dadd_rn(u0, __dmul_rn(fdt, (double)a.dudt[i]));
    const double vn = __dadd_rn(v0, __dmul_rn(fdt, (double)a.dvdt[i]));
    const double utx = __dadd_rn(un, __dmul_rn((double)a.drx[i], idt));
    const double uty = __dadd_rn(vn, __dmul_rn((double)a.dry[i], idt));
    double xn = __dadd_rn(x0, __dmul_rn(fdt, utx));
    double yn = __dadd_rn(y0, __dmul_rn(fdt, uty));
    if (a.d.periodic[0]) {
        if (xn >= a.d.hi[0])
            xn = __dsub_rn(xn, a.d.L[0]);
        else if (xn < a.d.lo[0])
            xn = __dadd_rn(xn, a.d.L[0]);
    }
    if (a.d.periodic[1]) {
        if (yn >= a.d.hi[1])
            yn = __dsub_rn(yn, a.d.L[1]);
        else if (yn < a.d.lo[1])
            yn = __dadd_rn(yn, a.d.L[1]);
    }
    if (a.skin_err) {
        const double mx = min_image(a.d, 0, __dsub_rn(xn, x0));
        const double my = min_image(a.d, 1, __dsub_rn(yn, y0));
        const double lim = a.disp_lim * a.h[i];
        if (mx * mx + my * my > lim * lim) atomicOr(a.skin_err, 1);
    }
    double pn = __dadd_rn(p0, __dmul_rn(fdt, (double)a.dpdt[i]));
    double ur = un, vr = vn;
    if (a.sponge_w > 0.0) {
        // relaxation towards (U, 0, 0), strength (distance from the
        // sponge's downstream edge / width)^2
        const double s = (a.sponge_x1 - xn) / a.sponge_w;
        if (s > 0.0) {
            const double k = fmin(1.0, 10.0 * a.sponge_U * dt / a.sponge_w * s * s);
            ur = un + (a.sponge_U - un) * k;
            vr = vn - vn * k;
            pn = pn - pn * k;
        }
    }
    a.x[i] = xn;
    a.y[i] = yn;
    a.u[i] = ur;
    a.v[i] = vr;
    a.p[i] = pn;
}

template <typename R>
__global__ void k_pec(PecArgs<R> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    pec_at<R>(a, i);
}

// ---------------------------------------------------------- time step ----
// h > 0, so the IEEE bit patterns of h order like the values.
__global__ void k_min_h(int n, const double *__restrict__ h,
                        unsigned long long *out) {
    unsigned long long m = ~0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(h[i]);
        m = b < m ? b : m;
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t < m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

// Eq. timestep: dt = min(0.25 h_min/(U + c_s), 0.125 h_min^2/nu) into
// dt[0], 1 / dt into dt[1].
__device__ __forceinline__ void k_dt_body(const unsigned long long *hmin_bits,
                                          double U, double cs, double nu,
                                          double *dt, double *tacc, int nsteps) {
    const double hmin = __longlong_as_double((long long)*hmin_bits);
    double v = __dmul_rn(0.25, __ddiv_rn(hmin, __dadd_rn(U, cs)));
    if (nu > 0.0) {
        double w = __dmul_rn(0.125, __ddiv_rn(__dmul_rn(hmin, hmin), nu));
        if (w < v) v = w;
    }
    dt[0] = v;
    // its reciprocal: the per-particle (u~ - u) = dr / dt of pass B and the
    // PEC stages multiply by it (FP64 divisions are slow on this GPU)
    dt[1] = __ddiv_rn(1.0, v);
    if (tacc) {
        for (int s = 0; s < nsteps; ++s) *tacc = __dadd_rn(*tacc, v);
    }
}

__global__ void k_dt(const unsigned long long *hmin_bits, double U, double cs,
                     double nu, double *dt, double *tacc, int nsteps) {
    k_dt_body(hmin_bits, U, cs, nu, dt, tacc, nsteps);
}

// ---------------------------------------------------------- small utils --
__global__ void k_reset_bbox(int *bbox, uint32_t *level_mask) {
    int t = threadIdx.x;
    if (t < MAX_LEVELS * 4) bbox[t] = (t & 1) ? -1 : 0x7fffffff;
    if (t == 0) *level_mask = 0;
}

__global__ void k_to_float(int n, ConvList c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < c.k; ++a) c.dst[a][i] = (float)c.src[a][i];
}

__global__ void k_float_to_double(int n, const float *src, double *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// ------------------------------------------------------- batched phases --
// One persistent launch per phase over the work items of several
// instances (see BatchSpan): each block takes items with the grid's
// stride, reads the owning instance's argument block and runs the same
// per-particle body as the single-instance kernel, so an instance's
// results do not depend on the batch it ran in.
template <typename R, int T>
__global__ void __launch_bounds__(BATCH_THREADS)
    k_pass_a_batch(const PassAArgs<R> *__restrict__ args, BatchSpan sp) {
    const Team<T> tm;
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const PassAArgs<R> &a = args[q];
        const int i = (item - __ldg(&sp.first[q])) * batch_rows(T) + (int)threadIdx.x / T;
        if (i < a.n) pass_a_at<R, T>(a, i, tm);
    }
}

template <typename R, int T>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(R) == 4 ? 5 : 1)
    k_pass_b_batch(const PassBArgs<R> *__restrict__ args, BatchSpan sp) {
    const Team<T> tm;
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const PassBArgs<R> &a = args[q];
        const int i = (item - __ldg(&sp.first[q])) * batch_rows(T) + (int)threadIdx.x / T;
        if (i < a.n) pass_b_at<R, T>(a, i, tm);
    }
}

template <int T>
__global__ void __launch_bounds__(BATCH_THREADS)
    k_wall_bc_batch(const WallBcArgs *__restrict__ args, BatchSpan sp) {
    const Team<T> tm;
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const WallBcArgs &a = args[q];
        const int k = (item - __ldg(&sp.first[q])) * batch_rows(T) + (int)threadIdx.x / T;
        if (k < a.w.n) wall_bc_at<T>(a, k, tm);
    }
}

template <typename R>
__global__ void __launch_bounds__(BATCH_THREADS)
    k_pec_batch(const PecArgs<R> *__restrict__ args, BatchSpan sp) {
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const PecArgs<R> &a = args[q];
        const int i = (item - __ldg(&sp.first[q])) * BATCH_THREADS + (int)threadIdx.x;
        if (i < a.n) pec_at<R>(a, i);
    }
}

__global__ void __launch_bounds__(BATCH_THREADS)
    k_rho_store_batch(const RhoStoreArgs *__restrict__ args, BatchSpan sp) {
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const RhoStoreArgs &a = args[q];
        const int i = (item - __ldg(&sp.first[q])) * BATCH_THREADS + (int)threadIdx.x;
        if (i < a.n) a.dst[i] = (double)a.src[i];
    }
}

// ------------------------------------------------------------- launchers --
static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

// Blocks of a persistent launch: what the GPU holds at once (resident
// blocks per SM by the kernel's occupancy, times the SMs), at most one
// per work item.
int gpu_sms() {
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            v = 1;
        return v > 0 ? v : 1;
    }();
    return sms;
}
template <class K>
static int persistent_blocks(K kernel, int total) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BATCH_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long g = (long long)per_sm * gpu_sms();
    return (int)(g < total ? g : total);
}

template <typename R>
void launch_pass_a_batch(cudaStream_t s, int team, const PassAArgs<R> *args,
                         const BatchSpan &sp) {
    if (sp.total <= 0) return;
    with_team_or(team, 1 << 30, [&](auto t) {
        constexpr int T = decltype(t)::value;
        auto k = k_pass_a_batch<R, T>;
        static const int g = persistent_blocks(k, 1 << 30);
        k<<<std::min(g, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
    });
}
template <typename R>
void launch_pass_b_batch(cudaStream_t s, int team, const PassBArgs<R> *args,
                         const BatchSpan &sp) {
    if (sp.total <= 0) return;
    with_team_or(team, 1 << 30, [&](auto t) {
        constexpr int T = decltype(t)::value;
        auto k = k_pass_b_batch<R, T>;
        static const int g = persistent_blocks(k, 1 << 30);
        k<<<std::min(g, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
    });
}
void launch_wall_bc_batch(cudaStream_t s, int team, const WallBcArgs *args,
                          const BatchSpan &sp) {
    if (sp.total <= 0) return;
    with_team_or(team, 1 << 30, [&](auto t) {
        constexpr int T = decltype(t)::value;
        auto k = k_wall_bc_batch<T>;
        static const int g = persistent_blocks(k, 1 << 30);
        k<<<std::min(g, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
    });
}
template <typename R>
void launch_pec_batch(cudaStream_t s, const PecArgs<R> *args, const BatchSpan &sp) {
    if (sp.total <= 0) return;
    static const int g = persistent_blocks(k_pec_batch<R>, 1 << 30);
    k_pec_batch<R><<<std::min(g, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
}
void launch_rho_store_batch(cudaStream_t s, const RhoStoreArgs *args, const BatchSpan &sp) {
    if (sp.total <= 0) return;
    static const int g = persistent_blocks(k_rho_store_batch, 1 << 30);
    k_rho_store_batch<<<std::min(g, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
}
template void launch_pass_a_batch<float>(cudaStream_t, int, const PassAArgs<float> *, const BatchSpan &);
template void launch_pass_a_batch<double>(cudaStream_t, int, const PassAArgs<double> *, const BatchSpan &);
template void launch_pass_b_batch<float>(cudaStream_t, int, const PassBArgs<float> *, const BatchSpan &);
template void launch_pass_b_batch<double>(cudaStream_t, int, const PassBArgs<double> *, const BatchSpan &);
template void launch_pec_batch<float>(cudaStream_t, const PecArgs<float> *, const BatchSpan &);
template void launch_pec_batch<double>(cudaStream_t, const PecArgs<double> *, const BatchSpan &);

template <typename R>
void launch_pass_a(cudaStream_t s, const PassAArgs<R> &a, int team) {
    if (a.n <= 0) return;
    with_team_or(team, a.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        if (a.w.n > 0)
            k_pass_a<R, T, true><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
        else
            k_pass_a<R, T, false><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
    });
}
template <typename R>
void launch_pass_b(cudaStream_t s, const PassBArgs<R> &a, int team) {
    if (a.n <= 0) return;
    with_team_or(team, a.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        if (a.w.n > 0)
            k_pass_b<R, T, true><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
        else
            k_pass_b<R, T, false><<<nblk(a.n * T, 128), 128, 0, s>>>(a);
    });
}
template <typename R>
void launch_pec(cudaStream_t s, const PecArgs<R> &a) {
    if (a.n > 0) k_pec<R><<<nblk(a.n, 256), 256, 0, s>>>(a);
}
template void launch_pass_a<double>(cudaStream_t, const PassAArgs<double> &, int);
template void launch_pass_a<float>(cudaStream_t, const PassAArgs<float> &, int);
template void launch_pass_b<double>(cudaStream_t, const PassBArgs<double> &, int);
template void launch_pass_b<float>(cudaStream_t, const PassBArgs<float> &, int);
template void launch_pec<double>(cudaStream_t, const PecArgs<double> &);
template void launch_pec<float>(cudaStream_t, const PecArgs<float> &);

template <typename R>
void launch_forces(cudaStream_t s, const ForceArgs<R> &a) {
    if (a.w.n <= 0) return;
    with_team(a.w.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_forces<R, T><<<nblk(a.w.n * T, 128), 128, 0, s>>>(a);
    });
}
template void launch_forces<double>(cudaStream_t, const ForceArgs<double> &);
template void launch_forces<float>(cudaStream_t, const ForceArgs<float> &);

void launch_wall_lists_count(cudaStream_t s, int n, const WallListArgs &a,
                             SortScratch &sc, int *launches) {
    if (n <= 0) return;
    if (a.w.n > 0) {
        with_team(a.w.n, [&](auto t) {
            constexpr int T = decltype(t)::value;
            k_wall_lists<T><<<nblk(a.w.n * T, 128), 128, 0, s>>>(a, 0);
        });
        *launches += 1;
    }
    exclusive_scan(s, a.cnt, (uint32_t *)a.off, n + 1, nullptr, sc, launches);
}

void launch_wall_lists_fill(cudaStream_t s, int n, const WallListArgs &a,
                            int *launches) {
    if (n <= 0 || a.w.n <= 0) return;
    with_team(a.w.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_wall_lists<T><<<nblk(a.w.n * T, 128), 128, 0, s>>>(a, 1);
    });
    sort_segments(s, n, a.off, a.list, a.cap, a.longq, a.nlong, launches);
    *launches += 1;
}

void launch_forces_total(cudaStream_t s, int nw, const double *fw,
                         const int64_t *id, double *out, double *total) {
    k_forces_total<<<1, 256, 0, s>>>(nw, fw, id, out, total);
}

void launch_wall_bc(cudaStream_t s, const WallBcArgs &a) {
    if (a.w.n <= 0) return;
    with_team(a.w.n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_wall_bc<T><<<nblk(a.w.n * T, 128), 128, 0, s>>>(a);
    });
}
void launch_nbr_ids(cudaStream_t s, int n, const uint32_t *off,
                    const uint32_t *list, const int64_t *id, int64_t *out) {
    if (n > 0) k_nbr_ids<<<nblk(n, 128), 128, 0, s>>>(n, off, list, id, out);
}
// One block: h_min and the time step together (small sets).
__device__ __forceinline__ void dt_small_at(int n, const double *__restrict__ h, double U,
                                            double cs, double nu,
                                            unsigned long long *hmin_bits, double *dt,
                                            double *tacc, int nsteps) {
    __shared__ unsigned long long wm[32];
    unsigned long long m = ~0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(h[i]);
        m = b < m ? b : m;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t < m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] < m ? wm[w] : m;
        *hmin_bits = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) k_dt_body(hmin_bits, U, cs, nu, dt, tacc, nsteps);
}

__global__ void __launch_bounds__(1024)
    k_dt_small(int n, const double *__restrict__ h, double U, double cs,
               double nu, unsigned long long *hmin_bits, double *dt,
               double *tacc, int nsteps) {
    dt_small_at(n, h, U, cs, nu, hmin_bits, dt, tacc, nsteps);
}

// The same for several small sets, one work item (block) each.
__global__ void __launch_bounds__(1024) k_dt_small_batch(const DtSmallRec *args, BatchSpan sp) {
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const DtSmallRec &r = args[sp.find(it)];
        dt_small_at(r.n, r.h, r.U, r.cs, r.nu, r.hmin_bits, r.dt, r.tacc, r.nsteps);
        __syncthreads();
    }
}
void launch_dt_small_batch(cudaStream_t s, const DtSmallRec *args, const BatchSpan &sp) {
    if (sp.total > 0)
        k_dt_small_batch<<<std::min(sp.total, 2 * gpu_sms()), 1024, 0, s>>>(args, sp);
}
int dt_small_max() { return 65536; }

int launch_dt(cudaStream_t s, int n, const double *h,
              unsigned long long *hmin_bits, double U, double cs, double nu,
              double *dt, double *tacc, int nsteps) {
    if (n <= dt_small_max()) {
        k_dt_small<<<1, 1024, 0, s>>>(n, h, U, cs, nu, hmin_bits, dt, tacc, nsteps);
        return 1;
    }
    cudaMemsetAsync(hmin_bits, 0xff, sizeof(unsigned long long), s);
    int blocks = nblk(n, 256);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_min_h<<<blocks, 256, 0, s>>>(n, h, hmin_bits);
    k_dt<<<1, 1, 0, s>>>(hmin_bits, U, cs, nu, dt, tacc, nsteps);
    return 2;
}
void launch_reset_bbox(cudaStream_t s, int *bbox, uint32_t *level_mask) {
    k_reset_bbox<<<1, MAX_LEVELS * 4, 0, s>>>(bbox, level_mask);
}
void launch_to_float(cudaStream_t s, int n, const ConvList &c) {
    if (n > 0 && c.k > 0) k_to_float<<<nblk(n, 256), 256, 0, s>>>(n, c);
}
void launch_float_to_double(cudaStream_t s, int n, const float *src,
                            double *dst) {
    if (n > 0) k_float_to_double<<<nblk(n, 256), 256, 0, s>>>(n, src, dst);
}

SPH_DEBUG_COUNTER(debug_failures_pairs)

}  // namespace sph
