// Background construction (section 3.3) and the fluid vorticity used by
// solution adaptivity.  Everything here runs in FP64: the background is
// built once at set-up and refreshed every few hundred steps, off the
// per-step path, and its decisions (marking, the Cr^3 test, the split
// threshold) are taken with explicitly rounded operations so that they
// match the definition bit for bit.
#include <algorithm>

#include "background.cuh"
#include "kernels.cuh"
#include "neighbors.cuh"
#include "team.cuh"

namespace sph {

template <int T>
__device__ __forceinline__ double team_max_d(unsigned mask, double v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
    return v;
}

template <int T>
__device__ __forceinline__ int team_any(unsigned mask, int v) {
    return T == 1 ? v : (__any_sync(mask, v) ? 1 : 0);
}

// --------------------------------------------------------------- omega --
template <int T>
__global__ void __launch_bounds__(128) k_vorticity(VortArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
    const double ui = a.u[i], vi = a.v[i];
    const double hinv = 1.0 / hi;
    double w = 0.0;
    for (uint32_t k = a.off[i] + tm.lane; k < a.off[i + 1]; k += T) {
        const int j = (int)a.list[k];
        if (j == i) continue;
        const double dx = min_image(a.d, 0, __dsub_rn(xi, a.x[j]));
        const double dy = min_image(a.d, 1, __dsub_rn(yi, a.y[j]));
        const double r = sqrt(dx * dx + dy * dy);
        if (!(r > 0.0)) continue;
        const double g = sigma_norm<double>() * hinv * hinv * hinv *
                         qs_dw<double>(r * hinv) / r;
        const double Vj = a.m[j] / a.rho[j];
        w += Vj * ((a.v[j] - vi) * (g * dx) - (a.u[j] - ui) * (g * dy));
    }
    w = team_sum<T>(tm.mask, w);
    if (tm.lane != 0) return;
    a.omega[i] = w;
    atomicMax(a.wmax, (unsigned long long)__double_as_longlong(fabs(w)));
}

// ---------------------------------------------------------------- mark --
// mark = 1 if a solid particle s (wall or region marker) has r < 3
// max(h_b, h_s); else 2 if the
// largest |omega_f| over fluid particles f with r < 3 max(h_b, h_f) exceeds
// vort_k max|omega|; else 0.  Candidates come from the cell grids of the
// solid and fluid sets, membership from the FP64 predicate.
template <int T>
__global__ void __launch_bounds__(128) k_bg_mark(BgMarkArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
    const float xr = (float)(xi - a.d.lo[0]), yr = (float)(yi - a.d.lo[1]);
    int hit = 0;
    if (a.nw > 0) {
        for_each_cell_team<T>(a.wg, a.d, 0, xr, yr, (float)hi, tm.lane, tm.mask,
                              [&](uint32_t s, uint32_t e) {
            for (uint32_t j = s + tm.lane; j < e && !hit; j += T)
                if (pred_fp64(a.d, xi, yi, hi, a.wx[j], a.wy[j], a.wh[j])) hit = 1;
        });
    }
    if (a.nr > 0) {
        for_each_cell_team<T>(a.rg, a.d, 0, xr, yr, (float)hi, tm.lane, tm.mask,
                              [&](uint32_t s, uint32_t e) {
            for (uint32_t j = s + tm.lane; j < e && !hit; j += T)
                if (pred_fp64(a.d, xi, yi, hi, a.rx[j], a.ry[j], a.rh[j])) hit = 1;
        });
    }
    int mk = team_any<T>(tm.mask, hit);
    if (!mk && a.nf > 0 && a.vort_k > 0.0) {
        const double wmax = __longlong_as_double((long long)*a.wmax);
        if (wmax > 0.0) {
            double pb = 0.0;
            for_each_cell_team<T>(a.fg, a.d, 0, xr, yr, (float)hi, tm.lane, tm.mask,
                                  [&](uint32_t s, uint32_t e) {
                for (uint32_t j = s + tm.lane; j < e; j += T)
                    if (pred_fp64(a.d, xi, yi, hi, a.fx[j], a.fy[j], a.fh[j]))
                        pb = fmax(pb, fabs(a.omega[j]));
            });
            pb = team_max_d<T>(tm.mask, pb);
            if (pb > __dmul_rn(a.vort_k, wmax)) mk = 2;
        }
    }
    if (tm.lane != 0) return;
    a.mark[i] = (uint32_t)mk;
    if (mk) {
        a.ds[i] = a.ds_min;
        atomicAdd(&a.counts[0], 1u);
        if (mk == 2) atomicAdd(&a.counts[1], 1u);
    }
}

// ---------------------------------------------------------------- size --
// Unmarked particles: over background neighbours j != i, lo / hi / g the
// least / largest / geometric-mean size; ds = Cr lo if hi / lo < Cr^3, else
// g; kept in [ds_min, ds_max]; unchanged without neighbours.  All
// particles: m_max = 1.05 rho0 ds^2, m_min = 0.5 rho0 ds^2.
template <int T>
__global__ void __launch_bounds__(128) k_bg_size(BgSizeArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    double d = a.ds[i];
    if (!a.mark[i]) {
        double lo = 1e308, hi = 0.0, slog = 0.0;
        int c = 0;
        for (uint32_t k = a.off[i] + tm.lane; k < a.off[i + 1]; k += T) {
            const int j = (int)a.list[k];
            if (j == i) continue;
            const double s = a.ds[j];
            lo = fmin(lo, s);
            hi = fmax(hi, s);
            slog += log(s);
            ++c;
        }
        lo = team_min<T>(tm.mask, lo);
        hi = team_max_d<T>(tm.mask, hi);
        slog = team_sum<T>(tm.mask, slog);
        c = team_sum<T>(tm.mask, c);
        if (c > 0)
            d = __ddiv_rn(hi, lo) < a.cr3 ? __dmul_rn(a.Cr, lo)
                                          : exp(__ddiv_rn(slog, (double)c));
        if (d > a.ds_max) d = a.ds_max;
        if (d < a.ds_min) d = a.ds_min;
    }
    if (tm.lane != 0) return;
    const double mref = __dmul_rn(__dmul_rn(a.rho0, d), d);
    a.ds_out[i] = d;
    a.mmax[i] = __dmul_rn(1.05, mref);
    a.mmin[i] = __dmul_rn(0.5, mref);
}

// ------------------------------------------------------------ h-smooth --
// Eq. h-smoothing over N(i), i included:
// h <- (1/2) ((h/2) (1 + sqrt(N_r / N_i)) + sum_j h_j / N_i).
template <int T>
__global__ void __launch_bounds__(128) k_bg_hsmooth(BgSmoothArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    double sh = 0.0;
    for (uint32_t k = a.off[i] + tm.lane; k < a.off[i + 1]; k += T)
        sh += a.h[a.list[k]];
    sh = team_sum<T>(tm.mask, sh);
    if (tm.lane != 0) return;
    const double Ni = (double)(a.off[i + 1] - a.off[i]);
    const double grow = __dadd_rn(1.0, __dsqrt_rn(__ddiv_rn(a.Nr, Ni)));
    a.h_out[i] = __dmul_rn(0.5, __dadd_rn(__dmul_rn(__dmul_rn(0.5, a.h[i]), grow),
                                          __ddiv_rn(sh, Ni)));
}

// -------------------------------------------------------------- minmax --
__global__ void k_minmax_pos(int n, const double *v, unsigned long long *out) {
    unsigned long long lo = ~0ull, hi = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v[i]);
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&out[0], lo);
        atomicMax(&out[1], hi);
    }
}

// ------------------------------------------------------------ launchers --
static inline int nblk(long long n, int bs) { return (int)((n + bs - 1) / bs); }

#define SPH_TEAM_LAUNCH(KER, n, args, s)                                      \
    with_team(n, [&](auto t_) {                                               \
        constexpr int T_ = decltype(t_)::value;                               \
        KER<T_><<<nblk((long long)(n) * T_, 128), 128, 0, s>>>(args);         \
    });

void launch_vorticity(cudaStream_t s, const VortArgs &a) {
    cudaMemsetAsync(a.wmax, 0, sizeof(unsigned long long), s);
    if (a.n <= 0) return;
    SPH_TEAM_LAUNCH(k_vorticity, a.n, a, s)
}

void launch_bg_mark(cudaStream_t s, const BgMarkArgs &a) {
    cudaMemsetAsync(a.counts, 0, 2 * sizeof(uint32_t), s);
    if (a.n <= 0) return;
    SPH_TEAM_LAUNCH(k_bg_mark, a.n, a, s)
}

void launch_bg_size(cudaStream_t s, const BgSizeArgs &a) {
    if (a.n <= 0) return;
    SPH_TEAM_LAUNCH(k_bg_size, a.n, a, s)
}

void launch_bg_hsmooth(cudaStream_t s, const BgSmoothArgs &a) {
    if (a.n <= 0) return;
    SPH_TEAM_LAUNCH(k_bg_hsmooth, a.n, a, s)
}

void launch_minmax_pos(cudaStream_t s, int n, const double *v,
                       unsigned long long *out) {
    cudaMemsetAsync(out, 0xff, sizeof(unsigned long long), s);
    cudaMemsetAsync(out + 1, 0, sizeof(unsigned long long), s);
    if (n <= 0) return;
    k_minmax_pos<<<std::min(nblk(n, 256), 608), 256, 0, s>>>(n, v, out);
}

#undef SPH_TEAM_LAUNCH

}  // namespace sph
