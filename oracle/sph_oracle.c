/*
 * Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see sph_oracle.h).
 *
 * Muta & Ramachandran, "Efficient and Accurate Adaptive Resolution for
 * Weakly-Compressible SPH", arXiv 2107.01276.  Section numbers and equation
 * labels below are the paper's.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no -ffast-math).
 * Per-particle sums run over N(i) in ascending neighbour index.  The
 * OpenMP loops are over independent particles only, so results do not
 * depend on the thread count.
 */
#include "sph_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846;
/* Point of inflection of the quintic spline in q (section 2.1, shifting). */
static const double XI_INFLECTION = 0.759298480738450;
static const int DIM = 2;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (timing only: every per-particle
 * sum runs in the same order whatever the count). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * Quintic spline, section 2, Eq. (kernel):
 *   W(q) = sigma2 [(3-q)^5 - 6(2-q)^5 + 15(1-q)^5]  for 0 <= q < 1
 *        = sigma2 [(3-q)^5 - 6(2-q)^5]               for 1 <= q < 2
 *        = sigma2 (3-q)^5                             for 2 <= q < 3
 *        = 0                                          for q >= 3
 * with sigma2 = 7 / (478 pi h^2), q = r / h.
 * dW/dr follows by differentiating each power: d/dq (a-q)^5 = -5 (a-q)^4.
 * ---------------------------------------------------------------------- */
static double p5(double a) { return a * a * a * a * a; }
static double p4(double a) { return a * a * a * a; }

static double w_of_q(double q) {
    if (q >= 3.0) return 0.0;
    double w = p5(3.0 - q);
    if (q < 2.0) w -= 6.0 * p5(2.0 - q);
    if (q < 1.0) w += 15.0 * p5(1.0 - q);
    return w;
}

static double dw_of_q(double q) {
    if (q >= 3.0) return 0.0;
    double w = -5.0 * p4(3.0 - q);
    if (q < 2.0) w += 30.0 * p4(2.0 - q);
    if (q < 1.0) w -= 75.0 * p4(1.0 - q);
    return w;
}

static double sigma2(double h) { return 7.0 / (478.0 * PI * h * h); }

double orc_W(double r, double h) { return sigma2(h) * w_of_q(r / h); }

double orc_dWdr(double r, double h) {
    return sigma2(h) / h * dw_of_q(r / h);
}

/* ------------------------------------------------------------------------
 * Neighbour predicate.  The gather sums of section 2 run over every j whose
 * kernel W(r_ij, h_i), W(r_ij, h_j) or W(r_ij, h_ij) is non-zero; with
 * support 3h that is r_ij < 3 max(h_i, h_j).  i itself is included.  On a
 * periodic axis the separation is the minimum image (section 2.2, periodic
 * ghosts give the same sets).
 * ---------------------------------------------------------------------- */
static double min_image(const orc_params *P, int axis, double d) {
    if (P->periodic[axis]) {
        double L = P->hi[axis] - P->lo[axis];
        double half = 0.5 * L;
        if (d > half)
            d -= L;
        else if (d < -half)
            d += L;
    }
    return d;
}

static void separation(const orc_params *P, double xi, double yi, double xj,
                       double yj, double *dx, double *dy) {
    *dx = min_image(P, 0, xi - xj);
    *dy = min_image(P, 1, yi - yj);
}

int orc_is_neighbor(const orc_params *P, double xi, double yi, double hi,
                    double xj, double yj, double hj) {
    double dx, dy;
    separation(P, xi, yi, xj, yj, &dx, &dy);
    double r2 = dx * dx + dy * dy;
    double R = 3.0 * (hi > hj ? hi : hj);
    return r2 < R * R;
}

long long orc_neighbors_brute(const orc_params *P, int n, const double *x,
                              const double *y, const double *h, int *off,
                              int *nbr, long long cap) {
    /* count pass */
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int j = 0; j < n; ++j)
            c += orc_is_neighbor(P, x[i], y[i], h[i], x[j], y[j], h[j]);
        cnt[i] = c;
    }
    long long tot = 0;
    for (int i = 0; i < n; ++i) {
        off[i] = (int)tot;
        tot += cnt[i];
    }
    off[n] = (int)tot;
    free(cnt);
    if (tot > cap) return tot;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        int k = off[i];
        for (int j = 0; j < n; ++j)
            if (orc_is_neighbor(P, x[i], y[i], h[i], x[j], y[j], h[j]))
                nbr[k++] = j;
    }
    return tot;
}

long long orc_neighbors_cross(const orc_params *P, int na, const double *xa,
                              const double *ya, const double *ha, int nb,
                              const double *xb, const double *yb,
                              const double *hb, int *off, int *nbr,
                              long long cap) {
    int *cnt = (int *)calloc((size_t)na + 1, sizeof(int));
#pragma omp parallel for schedule(dynamic, 64)
    for (int a = 0; a < na; ++a) {
        int c = 0;
        for (int b = 0; b < nb; ++b)
            c += orc_is_neighbor(P, xa[a], ya[a], ha[a], xb[b], yb[b], hb[b]);
        cnt[a] = c;
    }
    long long tot = 0;
    for (int a = 0; a < na; ++a) {
        off[a] = (int)tot;
        tot += cnt[a];
    }
    off[na] = (int)tot;
    free(cnt);
    if (tot > cap) return tot;
#pragma omp parallel for schedule(dynamic, 64)
    for (int a = 0; a < na; ++a) {
        int k = off[a];
        for (int b = 0; b < nb; ++b)
            if (orc_is_neighbor(P, xa[a], ya[a], ha[a], xb[b], yb[b], hb[b]))
                nbr[k++] = b;
    }
    return tot;
}

/* Uniform bucket grid with bucket side >= 3 h_max, so every neighbour of i
 * lies in the 3x3 buckets around i's bucket.  Same predicate as the brute
 * search; the lists are sorted ascending so the two agree entry by entry. */
static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

long long orc_neighbors_grid(const orc_params *P, int n, const double *x,
                             const double *y, const double *h, int *off,
                             int *nbr, long long cap) {
    if (n <= 0) {
        off[0] = 0;
        return 0;
    }
    double hmax = 0.0;
    for (int i = 0; i < n; ++i)
        if (h[i] > hmax) hmax = h[i];
    double side = 3.0 * hmax;
    int nc[2];
    double w[2];
    for (int a = 0; a < 2; ++a) {
        double L = P->hi[a] - P->lo[a];
        if (P->periodic[a]) {
            nc[a] = (int)floor(L / side);
            if (nc[a] < 1) nc[a] = 1;
            w[a] = L / nc[a];
        } else {
            nc[a] = (int)ceil(L / side);
            if (nc[a] < 1) nc[a] = 1;
            w[a] = side;
        }
    }
    long long ncell = (long long)nc[0] * nc[1];
    int *head = (int *)malloc((size_t)ncell * sizeof(int));
    int *next = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    int *cx = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    int *cy = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (long long c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = n - 1; i >= 0; --i) {
        int ix = (int)floor((x[i] - P->lo[0]) / w[0]);
        int iy = (int)floor((y[i] - P->lo[1]) / w[1]);
        if (ix < 0) ix = 0;
        if (ix > nc[0] - 1) ix = nc[0] - 1;
        if (iy < 0) iy = 0;
        if (iy > nc[1] - 1) iy = nc[1] - 1;
        cx[i] = ix;
        cy[i] = iy;
        long long c = (long long)iy * nc[0] + ix;
        next[i] = head[c];
        head[c] = i;
    }
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            long long tot = 0;
            for (int i = 0; i < n; ++i) {
                off[i] = (int)tot;
                tot += cnt[i];
            }
            off[n] = (int)tot;
            if (tot > cap) {
                free(cnt); free(head); free(next); free(cx); free(cy);
                return tot;
            }
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int k = (pass == 1) ? off[i] : 0;
            int c = 0;
            int xs[3], ys[3], nxs = 0, nys = 0;
            /* distinct bucket columns / rows within one bucket of i */
            for (int d = -1; d <= 1; ++d) {
                int a = cx[i] + d;
                if (P->periodic[0]) a = ((a % nc[0]) + nc[0]) % nc[0];
                if (a < 0 || a >= nc[0]) continue;
                int dup = 0;
                for (int t = 0; t < nxs; ++t) dup |= (xs[t] == a);
                if (!dup) xs[nxs++] = a;
            }
            for (int d = -1; d <= 1; ++d) {
                int b = cy[i] + d;
                if (P->periodic[1]) b = ((b % nc[1]) + nc[1]) % nc[1];
                if (b < 0 || b >= nc[1]) continue;
                int dup = 0;
                for (int t = 0; t < nys; ++t) dup |= (ys[t] == b);
                if (!dup) ys[nys++] = b;
            }
            for (int s = 0; s < nys; ++s)
                for (int r = 0; r < nxs; ++r)
                    for (int j = head[(long long)ys[s] * nc[0] + xs[r]];
                         j >= 0; j = next[j])
                        if (orc_is_neighbor(P, x[i], y[i], h[i], x[j], y[j],
                                            h[j])) {
                            if (pass == 1) nbr[k + c] = j;
                            ++c;
                        }
            if (pass == 0)
                cnt[i] = c;
            else
                qsort(nbr + k, (size_t)c, sizeof(int), cmp_int);
        }
    }
    long long tot = off[n];
    free(cnt); free(head); free(next); free(cx); free(cy);
    return tot;
}

/* ------------------------------------------------------------------------
 * Multi-level cell keys.  Definition (a build choice, the paper only asks
 * for a neighbour search that is rebuilt every iteration, section 3.4):
 *   level l_i: smallest l >= 0 with c0 2^l >= t where t = (3 h_i) / c0 in
 *              FP64; capped at the top level, whose cell spans the domain.
 *   per level and axis: cell side c_l = c0 2^l; on a periodic axis the
 *              count is max(1, floor(L / c_l)) and the width L / count,
 *              otherwise the count is max(1, ceil(L / c_l)), width c_l.
 *   cell index floor((x - lo) / width) clamped to [0, count - 1].
 *   key = l << 58 | morton(ix, iy), ix on the even bits.
 * ---------------------------------------------------------------------- */
int orc_max_level(const orc_params *P, double c0) {
    double Lmax = P->hi[0] - P->lo[0];
    double Ly = P->hi[1] - P->lo[1];
    if (Ly > Lmax) Lmax = Ly;
    int l = 0;
    while (ldexp(c0, l) < Lmax) ++l;
    return l;
}

static int level_of(double h, double c0, int lmax) {
    double t = (3.0 * h) / c0;
    int l;
    if (t <= 1.0) {
        l = 0;
    } else {
        int e;
        double f = frexp(t, &e); /* t = f 2^e, f in [0.5, 1) */
        l = (f == 0.5) ? e - 1 : e;
    }
    return l > lmax ? lmax : l;
}

static void level_grid(const orc_params *P, double c0, int l, int axis,
                       long long *count, double *width) {
    double L = P->hi[axis] - P->lo[axis];
    double c = ldexp(c0, l);
    long long nc;
    if (P->periodic[axis]) {
        nc = (long long)floor(L / c);
        if (nc < 1) nc = 1;
        *width = L / (double)nc;
    } else {
        nc = (long long)ceil(L / c);
        if (nc < 1) nc = 1;
        *width = c;
    }
    *count = nc;
}

static uint64_t spread_bits(uint64_t v) {
    /* bit k of v goes to bit 2k, plain loop */
    uint64_t out = 0;
    for (int k = 0; k < 29; ++k)
        if (v & (1ULL << k)) out |= 1ULL << (2 * k);
    return out;
}

void orc_cell_keys(const orc_params *P, double c0, int n, const double *x,
                   const double *y, const double *h, uint64_t *key,
                   int *level) {
    int lmax = orc_max_level(P, c0);
    for (int i = 0; i < n; ++i) {
        int l = level_of(h[i], c0, lmax);
        long long cnt[2];
        double w[2];
        level_grid(P, c0, l, 0, &cnt[0], &w[0]);
        level_grid(P, c0, l, 1, &cnt[1], &w[1]);
        long long ix = (long long)floor((x[i] - P->lo[0]) / w[0]);
        long long iy = (long long)floor((y[i] - P->lo[1]) / w[1]);
        if (ix < 0) ix = 0;
        if (ix > cnt[0] - 1) ix = cnt[0] - 1;
        if (iy < 0) iy = 0;
        if (iy > cnt[1] - 1) iy = cnt[1] - 1;
        key[i] = ((uint64_t)l << 58) | spread_bits((uint64_t)ix) |
                 (spread_bits((uint64_t)iy) << 1);
        if (level) level[i] = l;
    }
}


/* ------------------------------------------------------------------------
 * Dummy wall particles (section 2.2, Adami et al.).  For wall particle w,
 * over fluid neighbours f (r_wf < 3 max(h_w, h_f)), with
 * W_wf = W(r_wf, (h_w + h_f)/2):
 *   u^_w = sum u_f W_wf / sum W_wf                        (Eq. shepard)
 *   u_w  = 2 u_wall - u^_w                                (Eq. bc-wall)
 *   p_w  = sum p_f W_wf / sum W_wf                        (Eq. bc-pre, g = a_w = 0)
 * and p_w = 0, u^ = 0 without fluid neighbours.  Walls join the fluid's
 * sums as neighbours: mass m_w in the density, beta, p_avg and shifting
 * sums; in pass B, the prescribed wall velocity in the divergence term
 * (no penetration), the extrapolated velocity in the viscous term
 * (no slip), p_w in the pressure terms, with rho_w = rho0 and beta_w = 1.
 * Walls have no rates of their own.
 * ---------------------------------------------------------------------- */
static int g_nw = 0;
static double *g_w = NULL;   /* x, y, h, m, uw, vw, pw, ugx, ugy */
/* When set, pass B also writes each fluid particle's wall terms:
 * {pressure x, y, viscous x, y} of its momentum rate (test instrumentation
 * for the force balance below). */
static double *g_wall_acc = NULL;

void orc_record_wall_terms(double *acc) { g_wall_acc = acc; }

void orc_set_walls(int n, const double *x, const double *y, const double *h,
                   const double *m, const double *uw, const double *vw) {
    free(g_w);
    g_w = NULL;
    g_nw = n > 0 ? n : 0;
    if (g_nw == 0) return;
    g_w = (double *)calloc((size_t)g_nw * 9, sizeof(double));
    memcpy(g_w, x, sizeof(double) * n);
    memcpy(g_w + n, y, sizeof(double) * n);
    memcpy(g_w + 2 * n, h, sizeof(double) * n);
    memcpy(g_w + 3 * n, m, sizeof(double) * n);
    if (uw) memcpy(g_w + 4 * n, uw, sizeof(double) * n);
    if (vw) memcpy(g_w + 5 * n, vw, sizeof(double) * n);
}

#define WX(k) g_w[(k)]
#define WY(k) g_w[g_nw + (k)]
#define WH(k) g_w[2 * g_nw + (k)]
#define WM(k) g_w[3 * g_nw + (k)]
#define WU(k) g_w[4 * g_nw + (k)]
#define WV(k) g_w[5 * g_nw + (k)]
#define WP(k) g_w[6 * g_nw + (k)]
#define WGX(k) g_w[7 * g_nw + (k)]
#define WGY(k) g_w[8 * g_nw + (k)]

void orc_wall_bc(const orc_params *P, const orc_state *s, double *pw,
                 double *ugx, double *ugy) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int w = 0; w < g_nw; ++w) {
        double sw = 0.0, su = 0.0, sv = 0.0, sp = 0.0;
        for (int f = 0; f < s->n; ++f) {
            if (!orc_is_neighbor(P, WX(w), WY(w), WH(w), s->x[f], s->y[f],
                                 s->h[f]))
                continue;
            double dx, dy;
            separation(P, WX(w), WY(w), s->x[f], s->y[f], &dx, &dy);
            double W = orc_W(sqrt(dx * dx + dy * dy), 0.5 * (WH(w) + s->h[f]));
            sw += W;
            su += s->u[f] * W;
            sv += s->v[f] * W;
            sp += s->p[f] * W;
        }
        double uh = 0.0, vh = 0.0, p = 0.0;
        if (sw > 0.0) {
            uh = su / sw;
            vh = sv / sw;
            p = sp / sw;
        }
        pw[w] = p;
        ugx[w] = 2.0 * WU(w) - uh;
        ugy[w] = 2.0 * WV(w) - vh;
    }
}

static void wall_bc_update(const orc_params *P, const orc_state *s) {
    if (g_nw > 0)
        orc_wall_bc(P, s, &WP(0), &WGX(0), &WGY(0));
}

void orc_wall_bc_store(const orc_params *P, const orc_state *s) {
    wall_bc_update(P, s);
}

/* Wall neighbours of fluid particle i, ascending wall index. */
static int wall_nbrs(const orc_params *P, double xi, double yi, double hi,
                     int *out, int cap) {
    int c = 0;
    for (int w = 0; w < g_nw; ++w)
        if (orc_is_neighbor(P, xi, yi, hi, WX(w), WY(w), WH(w))) {
            if (c < cap) out[c] = w;
            ++c;
        }
    return c;
}

/* ------------------------------------------------------------------------
 * Pass A: summation density (section 2, Eq. sd-gather), variable-h
 * correction beta (Eq. beta), average pressure (Eq. pavg, N_i counts i
 * itself) and the limited shifting displacement (section 2.1, Eqs.
 * shift-deltar and shift-limit).
 *
 * Readings: the shifting denominator W(dx, xi h_ij) is taken as the kernel
 * at its inflection point for smoothing length h_ij = (h_i + h_j)/2, i.e.
 * W(xi h_ij, h_ij), and grad W_ij as grad_i W(r_ij, h_ij).  At r = 0 the
 * gradient is zero.  A particle whose beta is zero (no neighbour at r > 0)
 * gets no shift, and pass B gives it zero rates.
 * Returns the number of particles with beta == 0.
 * ---------------------------------------------------------------------- */
int orc_pass_a(const orc_params *P, int n, const double *x, const double *y,
               const double *h, const double *m, const double *p,
               const int *off, const int *nbr, orc_rhs_out *o) {
    const double w_xi = w_of_q(XI_INFLECTION);
    int degenerate = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : degenerate)
    for (int i = 0; i < n; ++i) {
        double rho = 0.0, srw = 0.0, psum = 0.0, spabs = 0.0;
        double ax = 0.0, ay = 0.0, sax = 0.0, say = 0.0;
        int cnt = 0;
        for (int k = off[i]; k < off[i + 1]; ++k) {
            int j = nbr[k];
            double dx, dy;
            separation(P, x[i], y[i], x[j], y[j], &dx, &dy);
            double r = sqrt(dx * dx + dy * dy);
            rho += m[j] * orc_W(r, h[i]);
            srw += m[j] * r * orc_dWdr(r, h[i]);
            psum += p[j];
            spabs += fabs(p[j]);
            cnt += 1;
            if (j != i && r > 0.0) {
                double hb = 0.5 * (h[i] + h[j]);
                double ratio = w_of_q(r / hb) / w_xi;
                double f = (m[j] / P->rho0) * (1.0 + 0.24 * p4(ratio)) *
                           orc_dWdr(r, hb) / r;
                ax += f * dx;
                ay += f * dy;
                sax += fabs(f * dx);
                say += fabs(f * dy);
            }
        }
        double wpx = 0, wpy = 0, wvx = 0, wvy = 0;   /* the walls' share */
        if (g_nw > 0) {
            int wl[2048];
            int nwl = wall_nbrs(P, x[i], y[i], h[i], wl, 2048);
            if (nwl > 2048) nwl = 2048;
            for (int k = 0; k < nwl; ++k) {
                int w = wl[k];
                double dx, dy;
                separation(P, x[i], y[i], WX(w), WY(w), &dx, &dy);
                double r = sqrt(dx * dx + dy * dy);
                rho += WM(w) * orc_W(r, h[i]);
                srw += WM(w) * r * orc_dWdr(r, h[i]);
                psum += WP(w);
                spabs += fabs(WP(w));
                cnt += 1;
                if (r > 0.0) {
                    double hb = 0.5 * (h[i] + WH(w));
                    double ratio = w_of_q(r / hb) / w_xi;
                    double f = (WM(w) / P->rho0) * (1.0 + 0.24 * p4(ratio)) *
                               orc_dWdr(r, hb) / r;
                    ax += f * dx;
                    ay += f * dy;
                    sax += fabs(f * dx);
                    say += fabs(f * dy);
                }
            }
        }
        double beta = -srw / (rho * DIM);
        o->rho[i] = rho;
        o->beta[i] = beta;
        o->pavg[i] = psum / cnt;
        o->nnb[i] = cnt;
        o->s_rho[i] = rho;
        o->s_beta[i] = fabs(beta);
        o->s_pavg[i] = spabs / cnt;
        double c = -0.5 * h[i] * h[i];
        double drx = c * ax, dry = c * ay;
        if (beta == 0.0) {
            drx = 0.0;
            dry = 0.0;
            degenerate += 1;
        }
        double mag = sqrt(drx * drx + dry * dry);
        double lim = 0.25 * h[i];
        if (mag > lim) {
            double theta = lim / mag;
            drx *= theta;
            dry *= theta;
        }
        o->drx[i] = drx;
        o->dry[i] = dry;
        o->s_drx[i] = 0.5 * h[i] * h[i] * sax;
        o->s_dry[i] = 0.5 * h[i] * h[i] * say;
    }
    return degenerate;
}

/* ------------------------------------------------------------------------
 * Pass B: EDAC pressure rate (section 2, Eq. edac:sph) and momentum rate
 * (Eq. mom-sph without the A_i/A_j stresses and third line, which the
 * paper's remark in section 2 says are not used), with
 *   P_i = (p_i - p_avg,i) / (rho_i^2 beta_i)                (Eq. mom:pre)
 *   grad W(r_ij, h_ij) = (grad W(h_i) + grad W(h_j)) / 2    (Eq. dw-avg)
 *   nu_e,i = alpha_e c_s h_i / 8,                           (Eq. edac-alpha)
 *   nu_e,ij = 4 nu_e,i nu_e,j / (nu_e,i + nu_e,j)           (Eq. nu-cleary)
 *   eta = 0.001 h_i^2,  (u~_i - u_i) = dr_i / dt            (Eq. shift-tvf)
 * Readings:
 *   pavg_mode 0: P_j uses p_avg,i, so a constant pressure offset cancels
 *     and a linear field gives grad p / rho (literal P_j with p_avg,j
 *     cancels a linear field to zero force); pavg_mode 1 is literal.
 *   edac_diff_denominator 1: the pressure-diffusion sum is divided by
 *     (r^2 + eta) like the viscous sum, which makes it nu_e lap p.
 *   edac_rho_factor 1: the third sum, an estimate of (u~ - u).grad p / rho,
 *     is multiplied by rho_i to match the continuum Eq. edac-corr.
 * Sums run over j != i (every term vanishes at j == i).
 * ---------------------------------------------------------------------- */
void orc_pass_b(const orc_params *P, double dt, int n, const double *x,
                const double *y, const double *h, const double *m,
                const double *p, const double *u, const double *v,
                const int *off, const int *nbr, orc_rhs_out *o) {
    const double c2 = P->cs * P->cs;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double beta_i = o->beta[i];
        if (beta_i == 0.0) {
            o->dpdt[i] = o->dudt[i] = o->dvdt[i] = 0.0;
            o->s_dpdt[i] = o->s_dudt[i] = o->s_dvdt[i] = 0.0;
            if (g_wall_acc)
                g_wall_acc[4 * i] = g_wall_acc[4 * i + 1] =
                    g_wall_acc[4 * i + 2] = g_wall_acc[4 * i + 3] = 0.0;
            continue;
        }
        double rho_i = o->rho[i];
        double pavg_i = o->pavg[i];
        double Pi = (p[i] - pavg_i) / (rho_i * rho_i * beta_i);
        double Pi_abs = (fabs(p[i]) + fabs(pavg_i)) /
                        (rho_i * rho_i * fabs(beta_i));
        double nu_i = P->alpha_e * P->cs * h[i] / 8.0;
        double eta = 0.001 * h[i] * h[i];
        double dux = o->drx[i] / dt, duy = o->dry[i] / dt;
        double div = 0, diff = 0, tvf = 0, ax = 0, ay = 0, vx = 0, vy = 0;
        double s_div = 0, s_diff = 0, s_tvf = 0, s_ax = 0, s_ay = 0,
               s_v = 0, s_vx = 0, s_vy = 0;
        (void)s_v;
        for (int k = off[i]; k < off[i + 1]; ++k) {
            int j = nbr[k];
            if (j == i) continue;
            double dx, dy;
            separation(P, x[i], y[i], x[j], y[j], &dx, &dy);
            double r2 = dx * dx + dy * dy;
            double r = sqrt(r2);
            double gi = 0.0, gj = 0.0;
            if (r > 0.0) {
                gi = orc_dWdr(r, h[i]) / r;
                gj = orc_dWdr(r, h[j]) / r;
            }
            double gWix = gi * dx, gWiy = gi * dy;
            double gWjx = gj * dx, gWjy = gj * dy;
            double gbar = 0.5 * (gi + gj);
            double rdotgbar = gbar * r2; /* r_ij . gradW(r_ij, h_ij) */
            double rho_j = o->rho[j], beta_j = o->beta[j];
            double Vj = m[j] / rho_j;
            double uij = u[i] - u[j], vij = v[i] - v[j];
            double pref = (P->pavg_mode == 0) ? pavg_i : o->pavg[j];
            double Pj = (p[j] - pref) / (rho_j * rho_j * beta_j);
            double Pj_abs = (fabs(p[j]) + fabs(pref)) /
                            (rho_j * rho_j * fabs(beta_j));
            double nu_j = P->alpha_e * P->cs * h[j] / 8.0;
            double nu_ij = 4.0 * nu_i * nu_j / (nu_i + nu_j);
            double dden = P->edac_diff_denominator ? (r2 + eta) : 1.0;

            div += Vj * (uij * gWix + vij * gWiy);
            diff += Vj * nu_ij * (p[i] - p[j]) * rdotgbar / dden;
            double fx = Pi * gWix + Pj * gWjx;
            double fy = Pi * gWiy + Pj * gWjy;
            tvf += m[j] * (dux * fx + duy * fy);
            ax -= m[j] * fx;
            ay -= m[j] * fy;
            double visc = m[j] * (4.0 * P->nu / (rho_i + rho_j)) * rdotgbar /
                          (r2 + eta);
            vx += visc * uij;
            vy += visc * vij;

            double au = fabs(u[i]) + fabs(u[j]), av = fabs(v[i]) + fabs(v[j]);
            s_div += Vj * (au * fabs(gWix) + av * fabs(gWiy));
            s_diff += Vj * nu_ij * (fabs(p[i]) + fabs(p[j])) * fabs(rdotgbar) /
                      dden;
            double afx = Pi_abs * fabs(gWix) + Pj_abs * fabs(gWjx);
            double afy = Pi_abs * fabs(gWiy) + Pj_abs * fabs(gWjy);
            s_tvf += m[j] * (fabs(dux) * afx + fabs(duy) * afy);
            s_ax += m[j] * afx;
            s_ay += m[j] * afy;
            s_vx += fabs(visc) * au;
            s_vy += fabs(visc) * av;
        }
        double wpx = 0, wpy = 0, wvx = 0, wvy = 0;   /* the walls' share */
        if (g_nw > 0) {
            int wl[2048];
            int nwl = wall_nbrs(P, x[i], y[i], h[i], wl, 2048);
            if (nwl > 2048) nwl = 2048;
            for (int k = 0; k < nwl; ++k) {
                int w = wl[k];
                double dx, dy;
                separation(P, x[i], y[i], WX(w), WY(w), &dx, &dy);
                double r2 = dx * dx + dy * dy;
                double r = sqrt(r2);
                double gi = 0.0, gj = 0.0;
                if (r > 0.0) {
                    gi = orc_dWdr(r, h[i]) / r;
                    gj = orc_dWdr(r, WH(w)) / r;
                }
                double gWix = gi * dx, gWiy = gi * dy;
                double gWjx = gj * dx, gWjy = gj * dy;
                double rdotgbar = 0.5 * (gi + gj) * r2;
                double Vj = WM(w) / P->rho0;
                /* prescribed wall velocity: no penetration */
                double uij = u[i] - WU(w), vij = v[i] - WV(w);
                double pref = (P->pavg_mode == 0) ? pavg_i : 0.0;
                double Pj = (WP(w) - pref) / (P->rho0 * P->rho0);
                double Pj_abs = (fabs(WP(w)) + fabs(pref)) / (P->rho0 * P->rho0);
                double nu_j = P->alpha_e * P->cs * WH(w) / 8.0;
                double nu_ij = 4.0 * nu_i * nu_j / (nu_i + nu_j);
                double dden = P->edac_diff_denominator ? (r2 + eta) : 1.0;
                div += Vj * (uij * gWix + vij * gWiy);
                diff += Vj * nu_ij * (p[i] - WP(w)) * rdotgbar / dden;
                double fx = Pi * gWix + Pj * gWjx;
                double fy = Pi * gWiy + Pj * gWjy;
                tvf += WM(w) * (dux * fx + duy * fy);
                ax -= WM(w) * fx;
                ay -= WM(w) * fy;
                wpx -= WM(w) * fx;
                wpy -= WM(w) * fy;
                /* extrapolated wall velocity: no slip */
                double ug = u[i] - WGX(w), vg = v[i] - WGY(w);
                double visc = WM(w) * (4.0 * P->nu / (rho_i + P->rho0)) *
                              rdotgbar / (r2 + eta);
                vx += visc * ug;
                vy += visc * vg;
                wvx += visc * ug;
                wvy += visc * vg;
                double au = fabs(u[i]) + fabs(WU(w)), av = fabs(v[i]) + fabs(WV(w));
                s_div += Vj * (au * fabs(gWix) + av * fabs(gWiy));
                s_diff += Vj * nu_ij * (fabs(p[i]) + fabs(WP(w))) *
                          fabs(rdotgbar) / dden;
                double afx = Pi_abs * fabs(gWix) + Pj_abs * fabs(gWjx);
                double afy = Pi_abs * fabs(gWiy) + Pj_abs * fabs(gWjy);
                s_tvf += WM(w) * (fabs(dux) * afx + fabs(duy) * afy);
                s_ax += WM(w) * afx;
                s_ay += WM(w) * afy;
                s_vx += fabs(visc) * (fabs(u[i]) + fabs(WGX(w)));
                s_vy += fabs(visc) * (fabs(v[i]) + fabs(WGY(w)));
            }
        }
        if (g_wall_acc) {
            g_wall_acc[4 * i] = wpx;
            g_wall_acc[4 * i + 1] = wpy;
            g_wall_acc[4 * i + 2] = wvx / beta_i;
            g_wall_acc[4 * i + 3] = wvy / beta_i;
        }
        double rf = P->edac_rho_factor ? rho_i : 1.0;
        o->dpdt[i] = (P->rho0 * c2 / beta_i) * div + diff / beta_i + rf * tvf;
        o->dudt[i] = ax + vx / beta_i;
        o->dvdt[i] = ay + vy / beta_i;
        double ab = fabs(beta_i);
        o->s_dpdt[i] = (P->rho0 * c2 / ab) * s_div + s_diff / ab + rf * s_tvf;
        o->s_dudt[i] = s_ax + s_vx / ab;
        o->s_dvdt[i] = s_ay + s_vy / ab;
    }
}

/* Section 2.4, Eq. timestep, with h_min over the fluid particles and U the
 * reference speed.  A zero viscosity drops the viscous limit. */
double orc_dt(const orc_params *P, int n, const double *h) {
    double hmin = DBL_MAX;
    for (int i = 0; i < n; ++i)
        if (h[i] < hmin) hmin = h[i];
    double dt = 0.25 * (hmin / (P->U_ref + P->cs));
    if (P->nu > 0.0) {
        double dv = 0.125 * (hmin * hmin / P->nu);
        if (dv < dt) dt = dv;
    }
    return dt;
}

static int *g_off = NULL, *g_nbr = NULL;
static long long g_cap = 0;
static int g_offn = 0;

static long long neighbors_auto(const orc_params *P, int n, const double *x,
                                const double *y, const double *h) {
    if (g_offn < n + 1) {
        free(g_off);
        g_off = (int *)malloc((size_t)(n + 1) * sizeof(int));
        g_offn = n + 1;
    }
    for (;;) {
        long long tot = orc_neighbors_grid(P, n, x, y, h, g_off, g_nbr, g_cap);
        if (tot <= g_cap) return tot;
        free(g_nbr);
        g_cap = tot + tot / 4 + 64;
        g_nbr = (int *)malloc((size_t)g_cap * sizeof(int));
    }
}

int orc_rhs(const orc_params *P, double dt, const orc_state *s,
            orc_rhs_out *o) {
    wall_bc_update(P, s);
    neighbors_auto(P, s->n, s->x, s->y, s->h);
    int deg = orc_pass_a(P, s->n, s->x, s->y, s->h, s->m, s->p, g_off, g_nbr,
                         o);
    orc_pass_b(P, dt, s->n, s->x, s->y, s->h, s->m, s->p, s->u, s->v, g_off,
               g_nbr, o);
    return deg;
}

/* ------------------------------------------------------------------------
 * Force on the solid, section "Force computation", Eq. force-sph: for each
 * wall particle w over its fluid neighbours j (r_wj < 3 max(h_w, h_j)),
 * r_wj = r_w - r_j and gradients with respect to r_w,
 *   f_p,w    = -m_w sum_j m_j (P_w grad W(r_wj, h_w) + P_j grad W(r_wj, h_j))
 *   f_visc,w =  m_w / beta_w sum_j m_j 4 nu / (rho_w + rho_j)
 *                 (r_wj . grad W_wj) / (|r_wj|^2 + eta_w) (u_w - u_j)
 * Reading F1: the pressures enter without the average-pressure offset,
 * P_w = p_w / rho0^2 and P_j = p_j / (rho_j^2 beta_j).  The offset takes a
 * constant out of a particle's own pressure gradient, harmless inside the
 * fluid, but the solid's sum runs over fluid on one side only, where the
 * pressure level itself is the load (with the offset a uniform pressure
 * would press on no wall).  The wall has rho_w = rho0, beta_w = 1, eta_w =
 * 0.001 h_w^2; grad W_wj is the mean of the two gradients (Eq. dw-avg) and
 * u_w the extrapolated (no-slip) wall velocity of the viscous sum.  p_w, u_w from the wall condition and
 * rho_j, beta_j from pass A, both at the given state.  out:
 * {f_p,x, f_p,y, f_visc,x, f_visc,y} summed over the walls in index order;
 * per_wall (NULL: not wanted) the four components of each wall particle.
 * ---------------------------------------------------------------------- */
void orc_forces(const orc_params *P, const orc_state *s, double *out,
                double *per_wall) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (g_nw == 0 || s->n == 0) return;
    wall_bc_update(P, s);
    neighbors_auto(P, s->n, s->x, s->y, s->h);
    const int n = s->n;
    orc_rhs_out o;
    double **arrs[] = {&o.rho, &o.beta, &o.pavg, &o.drx, &o.dry, &o.dpdt,
                       &o.dudt, &o.dvdt, &o.s_rho, &o.s_beta, &o.s_pavg,
                       &o.s_drx, &o.s_dry, &o.s_dpdt, &o.s_dudt, &o.s_dvdt};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k)
        *arrs[k] = (double *)calloc((size_t)n, sizeof(double));
    o.nnb = (int *)calloc((size_t)n, sizeof(int));
    orc_pass_a(P, n, s->x, s->y, s->h, s->m, s->p, g_off, g_nbr, &o);
    double *fw = (double *)calloc((size_t)g_nw * 4, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int w = 0; w < g_nw; ++w) {
        double fpx = 0, fpy = 0, fvx = 0, fvy = 0;
        const double eta = 0.001 * WH(w) * WH(w);
        for (int j = 0; j < n; ++j) {
            if (!orc_is_neighbor(P, WX(w), WY(w), WH(w), s->x[j], s->y[j],
                                 s->h[j]))
                continue;
            const double beta_j = o.beta[j];
            if (beta_j == 0.0) continue;
            double dx, dy;
            separation(P, WX(w), WY(w), s->x[j], s->y[j], &dx, &dy);
            const double r2 = dx * dx + dy * dy;
            const double r = sqrt(r2);
            double gw = 0.0, gj = 0.0;
            if (r > 0.0) {
                gw = orc_dWdr(r, WH(w)) / r;
                gj = orc_dWdr(r, s->h[j]) / r;
            }
            const double rho_j = o.rho[j];
            const double Pw = WP(w) / (P->rho0 * P->rho0);
            const double Pj = s->p[j] / (rho_j * rho_j * beta_j);
            fpx -= s->m[j] * (Pw * gw + Pj * gj) * dx;
            fpy -= s->m[j] * (Pw * gw + Pj * gj) * dy;
            const double rdotgbar = 0.5 * (gw + gj) * r2;
            const double visc = s->m[j] * (4.0 * P->nu / (P->rho0 + rho_j)) *
                                rdotgbar / (r2 + eta);
            fvx += visc * (WGX(w) - s->u[j]);
            fvy += visc * (WGY(w) - s->v[j]);
        }
        fw[4 * w] = WM(w) * fpx;
        fw[4 * w + 1] = WM(w) * fpy;
        fw[4 * w + 2] = WM(w) * fvx;   /* 1 / beta_w = 1 */
        fw[4 * w + 3] = WM(w) * fvy;
    }
    for (int w = 0; w < g_nw; ++w)
        for (int k = 0; k < 4; ++k) out[k] += fw[4 * w + k];
    if (per_wall) memcpy(per_wall, fw, sizeof(double) * 4 * (size_t)g_nw);
    free(fw);
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) free(*arrs[k]);
    free(o.nnb);
}

/* ------------------------------------------------------------------------
 * PEC integrator, section 2.4, Eqs. int-pre and int-cor.
 *   predict: u' = u0 + dt/2 a0; u~' = u' + dr0/dt; r' = r0 + dt/2 u~';
 *            p' = p0 + dt/2 (dp/dt)0
 *   correct: u = u0 + dt a'; u~ = u + dr'/dt; r = r0 + dt u~;
 *            p = p0 + dt (dp/dt)'
 * Positions are wrapped back into the box on periodic axes.
 * ---------------------------------------------------------------------- */
static double wrap(const orc_params *P, int axis, double x) {
    if (P->periodic[axis]) {
        double L = P->hi[axis] - P->lo[axis];
        if (x >= P->hi[axis])
            x -= L;
        else if (x < P->lo[axis])
            x += L;
    }
    return x;
}

static void pec_stage(const orc_params *P, double dt, double f, int n,
                      const double *x0, const double *y0, const double *u0,
                      const double *v0, const double *p0, const double *dudt,
                      const double *dvdt, const double *dpdt,
                      const double *drx, const double *dry, double *x,
                      double *y, double *u, double *v, double *p) {
    double fdt = f * dt;
    for (int i = 0; i < n; ++i) {
        double un = u0[i] + fdt * dudt[i];
        double vn = v0[i] + fdt * dvdt[i];
        double utx = un + drx[i] / dt;
        double uty = vn + dry[i] / dt;
        x[i] = wrap(P, 0, x0[i] + fdt * utx);
        y[i] = wrap(P, 1, y0[i] + fdt * uty);
        u[i] = un;
        v[i] = vn;
        p[i] = p0[i] + fdt * dpdt[i];
    }
}

void orc_pec_predict(const orc_params *P, double dt, int n, const double *x0,
                     const double *y0, const double *u0, const double *v0,
                     const double *p0, const double *dudt,
                     const double *dvdt, const double *dpdt,
                     const double *drx, const double *dry, double *x,
                     double *y, double *u, double *v, double *p) {
    pec_stage(P, dt, 0.5, n, x0, y0, u0, v0, p0, dudt, dvdt, dpdt, drx, dry,
              x, y, u, v, p);
}

void orc_pec_correct(const orc_params *P, double dt, int n, const double *x0,
                     const double *y0, const double *u0, const double *v0,
                     const double *p0, const double *dudt,
                     const double *dvdt, const double *dpdt,
                     const double *drx, const double *dry, double *x,
                     double *y, double *u, double *v, double *p) {
    pec_stage(P, dt, 1.0, n, x0, y0, u0, v0, p0, dudt, dvdt, dpdt, drx, dry,
              x, y, u, v, p);
}

typedef struct {
    double *buf;
    orc_rhs_out o;
} rhs_bufs;

static void rhs_bufs_init(rhs_bufs *b, int n) {
    int nn = n > 0 ? n : 1;
    b->buf = (double *)malloc((size_t)nn * 16 * sizeof(double));
    double *q = b->buf;
    b->o.rho = q; q += nn;
    b->o.beta = q; q += nn;
    b->o.pavg = q; q += nn;
    b->o.drx = q; q += nn;
    b->o.dry = q; q += nn;
    b->o.dpdt = q; q += nn;
    b->o.dudt = q; q += nn;
    b->o.dvdt = q; q += nn;
    b->o.s_rho = q; q += nn;
    b->o.s_beta = q; q += nn;
    b->o.s_pavg = q; q += nn;
    b->o.s_drx = q; q += nn;
    b->o.s_dry = q; q += nn;
    b->o.s_dpdt = q; q += nn;
    b->o.s_dudt = q; q += nn;
    b->o.s_dvdt = q; q += nn;
    b->o.nnb = (int *)malloc((size_t)nn * sizeof(int));
}

static void rhs_bufs_free(rhs_bufs *b) {
    free(b->buf);
    free(b->o.nnb);
}

int orc_step(const orc_params *P, orc_state *s, int nsteps, double *t) {
    int n = s->n;
    int nn = n > 0 ? n : 1;
    rhs_bufs a, b;
    rhs_bufs_init(&a, n);
    rhs_bufs_init(&b, n);
    double *x0 = (double *)malloc((size_t)nn * 5 * sizeof(double));
    double *y0 = x0 + nn, *u0 = y0 + nn, *v0 = u0 + nn, *p0 = v0 + nn;
    for (int st = 0; st < nsteps; ++st) {
        double dt = orc_dt(P, n, s->h);
        memcpy(x0, s->x, (size_t)n * sizeof(double));
        memcpy(y0, s->y, (size_t)n * sizeof(double));
        memcpy(u0, s->u, (size_t)n * sizeof(double));
        memcpy(v0, s->v, (size_t)n * sizeof(double));
        memcpy(p0, s->p, (size_t)n * sizeof(double));
        orc_rhs(P, dt, s, &a.o);
        orc_pec_predict(P, dt, n, x0, y0, u0, v0, p0, a.o.dudt, a.o.dvdt,
                        a.o.dpdt, a.o.drx, a.o.dry, s->x, s->y, s->u, s->v,
                        s->p);
        orc_rhs(P, dt, s, &b.o);
        orc_pec_correct(P, dt, n, x0, y0, u0, v0, p0, b.o.dudt, b.o.dvdt,
                        b.o.dpdt, b.o.drx, b.o.dry, s->x, s->y, s->u, s->v,
                        s->p);
        /* density is not integrated: keep the latest summation density */
        memcpy(s->rho, b.o.rho, (size_t)n * sizeof(double));
        *t += dt;
    }
    free(x0);
    rhs_bufs_free(&a);
    rhs_bufs_free(&b);
    return 0;
}

/* ========================================================================
 * Adaptive refinement, section 3.
 * ====================================================================== */

/* m_ref from the background (section 3.3): a fluid particle takes the
 * smallest background reference mass rho0 ds_b^2 over background particles
 * b with r_ib < 3 max(h_i, h_b); with none in range, the nearest background
 * particle's (ties to the lower index).  m_max = 1.05 m_ref,
 * m_min = 0.5 m_ref. */
void orc_bg_resolution(const orc_params *P, orc_state *s, int nb,
                       const double *bx, const double *by, const double *bh,
                       const double *bds) {
    if (nb <= 0) return;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < s->n; ++i) {
        double best = -1.0;
        double nr2 = DBL_MAX;
        int nearest = -1;
        for (int b = 0; b < nb; ++b) {
            double dx, dy;
            separation(P, s->x[i], s->y[i], bx[b], by[b], &dx, &dy);
            double r2 = dx * dx + dy * dy;
            double R = 3.0 * (s->h[i] > bh[b] ? s->h[i] : bh[b]);
            double mref = P->rho0 * bds[b] * bds[b];
            if (r2 < R * R && (best < 0.0 || mref < best)) best = mref;
            if (r2 < nr2) {
                nr2 = r2;
                nearest = b;
            }
        }
        if (best < 0.0) best = P->rho0 * bds[nearest] * bds[nearest];
        s->mmax[i] = 1.05 * best;
        s->mmin[i] = 0.5 * best;
    }
}

/* Hexagon directions k pi / 3, k = 0..5 (cosines and sines written out). */
static const double HEX_C[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
static const double HEX_S[6] = {0.0, 0.8660254037844386, 0.8660254037844386,
                                0.0, -0.8660254037844386, -0.8660254037844386};

typedef struct {
    long long id;
    int idx;
} id_idx;

static int cmp_id_idx(const void *a, const void *b) {
    long long x = ((const id_idx *)a)->id, y = ((const id_idx *)b)->id;
    return (x > y) - (x < y);
}

/* Split (section 3.1): a particle with m > m_max becomes 7 children, one
 * (m_max <= 0 means no limit: such a particle is never split or merged)
 * at the centre and six on the circle of radius eps h at angles k pi/3,
 * each with smoothing length alpha h and mass m/7 (the centre child takes
 * m - 6 (m/7) so the masses add up to m); rho, u, v, p, m_min, m_max are
 * copied.  The centre child keeps the parent's id and slot; the six others
 * are appended, and parent number r (counting parents in id order) gives
 * them ids next_id + 6 r + k. */
int orc_split(const orc_params *P, orc_state *s, long long *next_id) {
    int n = s->n;
    id_idx *par = (id_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(id_idx));
    int np = 0;
    for (int i = 0; i < n; ++i)
        if (s->mmax[i] > 0.0 && s->m[i] > s->mmax[i]) {
            par[np].id = s->id[i];
            par[np].idx = i;
            ++np;
        }
    if ((long long)n + 6LL * np > s->cap) {
        free(par);
        return -1;
    }
    qsort(par, (size_t)np, sizeof(id_idx), cmp_id_idx);
    for (int r = 0; r < np; ++r) {
        int i = par[r].idx;
        double m = s->m[i], h = s->h[i];
        double mc = m / 7.0;
        double rad = P->split_eps * h;
        for (int k = 0; k < 6; ++k) {
            int c = n + 6 * r + k;
            s->x[c] = wrap(P, 0, s->x[i] + rad * HEX_C[k]);
            s->y[c] = wrap(P, 1, s->y[i] + rad * HEX_S[k]);
            s->u[c] = s->u[i];
            s->v[c] = s->v[i];
            s->p[c] = s->p[i];
            s->rho[c] = s->rho[i];
            s->m[c] = mc;
            s->h[c] = P->split_alpha * h;
            s->mmin[c] = s->mmin[i];
            s->mmax[c] = s->mmax[i];
            s->id[c] = *next_id + 6LL * r + k;
        }
        s->m[i] = m - 6.0 * mc;
        s->h[i] = P->split_alpha * h;
    }
    s->n = n + 6 * np;
    *next_id += 6LL * np;
    free(par);
    return np;
}

/* Merge round (section 3.2).  i may merge with j != i in N(i) when neither
 * is to be split (m > m_max), r_ij < (h_i + h_j)/2 (tested as r^2 <
 * ((h_i + h_j)/2)^2) and m_i + m_j < max(m_max,i, m_max,j); closest_i is
 * the admissible j of least (r_ij^2, id_j).  Mutually closest pairs merge
 * into the one with the smaller id: mass m_a + m_b; position, velocity,
 * pressure and density mass-weighted (Eqs. merged-pos, merged-prop, with
 * b's periodic image nearest a); h from Eq. merged-h with d = 2; the kept
 * particle keeps its m_min, m_max.  The other particle is removed and the
 * survivors keep their relative order. */
int orc_merge_round(const orc_params *P, orc_state *s) {
    int n = s->n;
    if (n <= 1) return 0;
    neighbors_auto(P, n, s->x, s->y, s->h);
    int *closest = (int *)malloc((size_t)n * sizeof(int));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        closest[i] = -1;
        if (!(s->mmax[i] > 0.0) || s->m[i] > s->mmax[i]) continue;
        double br2 = 0.0;
        long long bid = 0;
        for (int k = g_off[i]; k < g_off[i + 1]; ++k) {
            int j = g_nbr[k];
            if (j == i || !(s->mmax[j] > 0.0) || s->m[j] > s->mmax[j]) continue;
            double dx, dy;
            separation(P, s->x[i], s->y[i], s->x[j], s->y[j], &dx, &dy);
            double r2 = dx * dx + dy * dy;
            double hh = 0.5 * (s->h[i] + s->h[j]);
            if (!(r2 < hh * hh)) continue;
            double mx = s->mmax[i] > s->mmax[j] ? s->mmax[i] : s->mmax[j];
            if (!(s->m[i] + s->m[j] < mx)) continue;
            if (closest[i] < 0 || r2 < br2 || (r2 == br2 && s->id[j] < bid)) {
                closest[i] = j;
                br2 = r2;
                bid = s->id[j];
            }
        }
    }
    const double W01 = orc_W(0.0, 1.0);
    char *dead = (char *)calloc((size_t)n, 1);
    int pairs = 0;
    for (int i = 0; i < n; ++i) {
        int j = closest[i];
        if (j < 0 || closest[j] != i || s->id[i] > s->id[j]) continue;
        /* i kept (smaller id), j removed */
        double ma = s->m[i], mb = s->m[j], mm = ma + mb;
        double xa = s->x[i], ya = s->y[i];
        double xb = xa + min_image(P, 0, s->x[j] - xa);
        double yb = ya + min_image(P, 1, s->y[j] - ya);
        double xm = (ma * xa + mb * xb) / mm;
        double ym = (ma * ya + mb * yb) / mm;
        double ra = sqrt((xm - xa) * (xm - xa) + (ym - ya) * (ym - ya));
        double rb = sqrt((xm - xb) * (xm - xb) + (ym - yb) * (ym - yb));
        double den = ma * orc_W(ra, s->h[i]) + mb * orc_W(rb, s->h[j]);
        double hm = sqrt(mm * W01 / den);
        s->u[i] = (ma * s->u[i] + mb * s->u[j]) / mm;
        s->v[i] = (ma * s->v[i] + mb * s->v[j]) / mm;
        s->p[i] = (ma * s->p[i] + mb * s->p[j]) / mm;
        s->rho[i] = (ma * s->rho[i] + mb * s->rho[j]) / mm;
        s->x[i] = wrap(P, 0, xm);
        s->y[i] = wrap(P, 1, ym);
        s->m[i] = mm;
        s->h[i] = hm;
        dead[j] = 1;
        ++pairs;
    }
    int w = 0;
    for (int i = 0; i < n; ++i) {
        if (dead[i]) continue;
        if (w != i) {
            s->x[w] = s->x[i]; s->y[w] = s->y[i]; s->u[w] = s->u[i];
            s->v[w] = s->v[i]; s->p[w] = s->p[i]; s->rho[w] = s->rho[i];
            s->m[w] = s->m[i]; s->h[w] = s->h[i]; s->mmin[w] = s->mmin[i];
            s->mmax[w] = s->mmax[i]; s->id[w] = s->id[i];
        }
        ++w;
    }
    s->n = w;
    free(dead);
    free(closest);
    return pairs;
}

/* Summation density (walls included), limited shift (Eqs. shift-deltar,
 * shift-limit, same readings as pass A, walls included) and the gradients
 * of the Taylor correction over fluid neighbours:
 * grad phi_i = sum_{j != i} V_j (phi_j - phi_i) grad_i W(r_ij, h_i) with
 * V_j = m_j / rho_j (the paper names no gradient operator; this is the
 * first-order form consistent with its gather sums). */
void orc_shift_compute(const orc_params *P, const orc_state *s, double *rho,
                       double *drx, double *dry, double *gux, double *guy,
                       double *gvx, double *gvy, double *gpx, double *gpy) {
    const double w_xi = w_of_q(XI_INFLECTION);
    int n = s->n;
    neighbors_auto(P, n, s->x, s->y, s->h);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double r_ = 0.0;
        for (int k = g_off[i]; k < g_off[i + 1]; ++k) {
            int j = g_nbr[k];
            double dx, dy;
            separation(P, s->x[i], s->y[i], s->x[j], s->y[j], &dx, &dy);
            r_ += s->m[j] * orc_W(sqrt(dx * dx + dy * dy), s->h[i]);
        }
        if (g_nw > 0) {
            int wl[2048];
            int nwl = wall_nbrs(P, s->x[i], s->y[i], s->h[i], wl, 2048);
            if (nwl > 2048) nwl = 2048;
            for (int k = 0; k < nwl; ++k) {
                double dx, dy;
                separation(P, s->x[i], s->y[i], WX(wl[k]), WY(wl[k]), &dx, &dy);
                r_ += WM(wl[k]) * orc_W(sqrt(dx * dx + dy * dy), s->h[i]);
            }
        }
        rho[i] = r_;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double ax = 0, ay = 0, ux = 0, uy = 0, vx = 0, vy = 0, px = 0, py = 0;
        for (int k = g_off[i]; k < g_off[i + 1]; ++k) {
            int j = g_nbr[k];
            if (j == i) continue;
            double dx, dy;
            separation(P, s->x[i], s->y[i], s->x[j], s->y[j], &dx, &dy);
            double r = sqrt(dx * dx + dy * dy);
            if (!(r > 0.0)) continue;
            double hb = 0.5 * (s->h[i] + s->h[j]);
            double ratio = w_of_q(r / hb) / w_xi;
            double f = (s->m[j] / P->rho0) * (1.0 + 0.24 * p4(ratio)) *
                       orc_dWdr(r, hb) / r;
            ax += f * dx;
            ay += f * dy;
            double g = orc_dWdr(r, s->h[i]) / r;
            double Vj = s->m[j] / rho[j];
            double du = s->u[j] - s->u[i], dv = s->v[j] - s->v[i],
                   dp = s->p[j] - s->p[i];
            ux += Vj * du * g * dx;
            uy += Vj * du * g * dy;
            vx += Vj * dv * g * dx;
            vy += Vj * dv * g * dy;
            px += Vj * dp * g * dx;
            py += Vj * dp * g * dy;
        }
        if (g_nw > 0) {
            int wl[2048];
            int nwl = wall_nbrs(P, s->x[i], s->y[i], s->h[i], wl, 2048);
            if (nwl > 2048) nwl = 2048;
            for (int k = 0; k < nwl; ++k) {
                int w = wl[k];
                double dx, dy;
                separation(P, s->x[i], s->y[i], WX(w), WY(w), &dx, &dy);
                double r = sqrt(dx * dx + dy * dy);
                if (!(r > 0.0)) continue;
                double hb = 0.5 * (s->h[i] + WH(w));
                double ratio = w_of_q(r / hb) / w_xi;
                double f = (WM(w) / P->rho0) * (1.0 + 0.24 * p4(ratio)) *
                           orc_dWdr(r, hb) / r;
                ax += f * dx;
                ay += f * dy;
            }
        }
        double c = -0.5 * s->h[i] * s->h[i];
        double sx = c * ax, sy = c * ay;
        double mag = sqrt(sx * sx + sy * sy);
        double lim = 0.25 * s->h[i];
        if (mag > lim) {
            double th = lim / mag;
            sx *= th;
            sy *= th;
        }
        drx[i] = sx;
        dry[i] = sy;
        gux[i] = ux; guy[i] = uy;
        gvx[i] = vx; gvy[i] = vy;
        gpx[i] = px; gpy[i] = py;
    }
}

void orc_shift_round(const orc_params *P, orc_state *s) {
    int n = s->n;
    int nn = n > 0 ? n : 1;
    double *b = (double *)malloc((size_t)nn * 9 * sizeof(double));
    double *rho = b, *drx = b + nn, *dry = b + 2 * nn, *gux = b + 3 * nn,
           *guy = b + 4 * nn, *gvx = b + 5 * nn, *gvy = b + 6 * nn,
           *gpx = b + 7 * nn, *gpy = b + 8 * nn;
    orc_shift_compute(P, s, rho, drx, dry, gux, guy, gvx, gvy, gpx, gpy);
    for (int i = 0; i < n; ++i) {
        s->x[i] = wrap(P, 0, s->x[i] + drx[i]);
        s->y[i] = wrap(P, 1, s->y[i] + dry[i]);
        s->u[i] = s->u[i] + (gux[i] * drx[i] + guy[i] * dry[i]);
        s->v[i] = s->v[i] + (gvx[i] * drx[i] + gvy[i] * dry[i]);
        s->p[i] = s->p[i] + (gpx[i] * drx[i] + gpy[i] * dry[i]);
        s->rho[i] = rho[i];
    }
    free(b);
}

/* h_i = hdx (mbar_i / rho_i)^(1/2): mbar_i the mean mass over the fluid
 * N(i) (i included), rho_i the summation density with walls (section 3.1, "h = C
 * (m/rho)^(1/d)" with the neighbourhood-average mass).  One evaluation. */
void orc_h_update(const orc_params *P, orc_state *s) {
    int n = s->n;
    int nn = n > 0 ? n : 1;
    double *hn = (double *)malloc((size_t)nn * 2 * sizeof(double));
    double *rn = hn + nn;
    neighbors_auto(P, n, s->x, s->y, s->h);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double rho = 0.0, msum = 0.0;
        int cnt = 0;
        for (int k = g_off[i]; k < g_off[i + 1]; ++k) {
            int j = g_nbr[k];
            double dx, dy;
            separation(P, s->x[i], s->y[i], s->x[j], s->y[j], &dx, &dy);
            rho += s->m[j] * orc_W(sqrt(dx * dx + dy * dy), s->h[i]);
            msum += s->m[j];
            cnt += 1;
        }
        if (g_nw > 0) {
            int wl[2048];
            int nwl = wall_nbrs(P, s->x[i], s->y[i], s->h[i], wl, 2048);
            if (nwl > 2048) nwl = 2048;
            for (int k = 0; k < nwl; ++k) {
                double dx, dy;
                separation(P, s->x[i], s->y[i], WX(wl[k]), WY(wl[k]), &dx, &dy);
                rho += WM(wl[k]) * orc_W(sqrt(dx * dx + dy * dy), s->h[i]);
            }
        }
        rn[i] = rho;
        hn[i] = P->hdx * sqrt((msum / cnt) / rho);
    }
    for (int i = 0; i < n; ++i) {
        s->h[i] = hn[i];
        s->rho[i] = rn[i];
    }
    free(hn);
}

/* One adaptation (section 3.4, steps ii-iii): resolution from the
 * background, one split pass, merge_iters merge rounds, shift_iters shift
 * rounds with Taylor correction, then the h update. */
int orc_adapt(const orc_params *P, orc_state *s, int nb, const double *bx,
              const double *by, const double *bh, const double *bds,
              long long *next_id, orc_adapt_stats *st) {
    orc_adapt_stats z;
    memset(&z, 0, sizeof(z));
    z.n_before = s->n;
    for (int i = 0; i < s->n; ++i) z.mass_before += s->m[i];
    orc_bg_resolution(P, s, nb, bx, by, bh, bds);
    int ns = orc_split(P, s, next_id);
    if (ns < 0) {
        if (st) *st = z;
        return -1;
    }
    z.n_split = ns;
    for (int r = 0; r < P->merge_iters; ++r) z.n_merged += orc_merge_round(P, s);
    for (int r = 0; r < P->shift_iters; ++r) orc_shift_round(P, s);
    orc_h_update(P, s);
    z.n_after = s->n;
    for (int i = 0; i < s->n; ++i) z.mass_after += s->m[i];
    if (st) *st = z;
    return 0;
}

/* ------------------------------------------------------------------------
 * Background particles, section 3.3.
 *
 * The background set defines the resolution field: each background
 * particle carries a size ds (its m_ref = rho0 ds^2), a mass m, a smoothing
 * length h and a persistent id.  One iteration of the construction:
 *   1. boundary marking: a background particle with a solid particle in
 *      range (r < 3 max(h_b, h_s)) takes ds = ds_min; with solution
 *      adaptivity also one whose phi (max |omega| over the fluid particles
 *      in range) exceeds vort_k max|omega|;
 *   2. size rule for the others over their background neighbours j != i
 *      (sizes after step 1): with lo, hi, g the least, largest and
 *      geometric-mean size, ds = Cr lo if hi / lo < Cr^3, else g; kept in
 *      [ds_min, ds_max]; no neighbour leaves ds unchanged.  Every particle
 *      reads the sizes of the same (previous) sweep;
 *   3. split of particles with m > 1.05 rho0 ds^2 into seven children as
 *      for the fluid (section 3.1), children copy ds;
 *   4. smooth_iters times: h-smoothing (Eq. h-smoothing, N_i and the sum
 *      of h_j over N(i) including i) and one shifting step (Eqs.
 *      shift-deltar, shift-limit with volumes m_j / rho0), both over the
 *      background set alone.
 * The whole construction repeats the iteration 3 ceil(log(ds_max/ds_min) /
 * log Cr) times (section 3.3).
 * ---------------------------------------------------------------------- */

/* Variable-h neighbour search for sets whose h spans a wide range: the
 * particles are grouped into classes of h (h / h_min in [2^k, 2^(k+1))),
 * each class bucketed with side >= 3 h_max of the class, and particle i
 * scans, per class, the buckets within 3 max(h_i, h_max of the class).
 * Same predicate and ascending order as orc_neighbors_brute. */
long long orc_neighbors_classes(const orc_params *P, int n, const double *x,
                                const double *y, const double *h, int *off,
                                int *nbr, long long cap) {
    if (n <= 0) {
        off[0] = 0;
        return 0;
    }
    double hmin = DBL_MAX;
    for (int i = 0; i < n; ++i)
        if (h[i] < hmin) hmin = h[i];
    enum { MAXC = 24 };
    int *cls = (int *)malloc((size_t)n * sizeof(int));
    int ncls = 0;
    for (int i = 0; i < n; ++i) {
        int e;
        frexp(h[i] / hmin, &e);   /* h/hmin in [2^(e-1), 2^e) */
        int k = e - 1;
        if (k < 0) k = 0;
        if (k > MAXC - 1) k = MAXC - 1;
        cls[i] = k;
        if (k + 1 > ncls) ncls = k + 1;
    }
    double chmax[MAXC];
    int nc[MAXC][2];
    double w[MAXC][2];
    int *head[MAXC];
    for (int k = 0; k < ncls; ++k) chmax[k] = 0.0;
    for (int i = 0; i < n; ++i)
        if (h[i] > chmax[cls[i]]) chmax[cls[i]] = h[i];
    int *next = (int *)malloc((size_t)n * sizeof(int));
    int *bx = (int *)malloc((size_t)n * sizeof(int));
    int *by = (int *)malloc((size_t)n * sizeof(int));
    for (int k = 0; k < ncls; ++k) {
        head[k] = NULL;
        if (chmax[k] <= 0.0) continue;
        double side = 3.0 * chmax[k];
        for (int a = 0; a < 2; ++a) {
            double L = P->hi[a] - P->lo[a];
            if (P->periodic[a]) {
                nc[k][a] = (int)floor(L / side);
                if (nc[k][a] < 1) nc[k][a] = 1;
                w[k][a] = L / nc[k][a];
            } else {
                nc[k][a] = (int)ceil(L / side);
                if (nc[k][a] < 1) nc[k][a] = 1;
                w[k][a] = side;
            }
        }
        long long ncell = (long long)nc[k][0] * nc[k][1];
        head[k] = (int *)malloc((size_t)ncell * sizeof(int));
        for (long long c = 0; c < ncell; ++c) head[k][c] = -1;
    }
    for (int i = n - 1; i >= 0; --i) {
        int k = cls[i];
        int ix = (int)floor((x[i] - P->lo[0]) / w[k][0]);
        int iy = (int)floor((y[i] - P->lo[1]) / w[k][1]);
        if (ix < 0) ix = 0;
        if (ix > nc[k][0] - 1) ix = nc[k][0] - 1;
        if (iy < 0) iy = 0;
        if (iy > nc[k][1] - 1) iy = nc[k][1] - 1;
        bx[i] = ix;
        by[i] = iy;
        long long c = (long long)iy * nc[k][0] + ix;
        next[i] = head[k][c];
        head[k][c] = i;
    }
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            long long tot = 0;
            for (int i = 0; i < n; ++i) {
                off[i] = (int)tot;
                tot += cnt[i];
            }
            off[n] = (int)tot;
            if (tot > cap) break;
        }
#pragma omp parallel for schedule(dynamic, 32)
        for (int i = 0; i < n; ++i) {
            int kbase = (pass == 1) ? off[i] : 0;
            int c = 0;
            for (int k = 0; k < ncls; ++k) {
                if (!head[k]) continue;
                double R = 3.0 * (h[i] > chmax[k] ? h[i] : chmax[k]);
                /* bucket of i in class k's grid */
                int ix = (int)floor((x[i] - P->lo[0]) / w[k][0]);
                int iy = (int)floor((y[i] - P->lo[1]) / w[k][1]);
                int sx = (int)ceil(R / w[k][0]) + 1, sy = (int)ceil(R / w[k][1]) + 1;
                int x0 = ix - sx, x1 = ix + sx, y0 = iy - sy, y1 = iy + sy;
                if (P->periodic[0] && x1 - x0 + 1 >= nc[k][0]) {
                    x0 = 0;
                    x1 = nc[k][0] - 1;
                }
                if (P->periodic[1] && y1 - y0 + 1 >= nc[k][1]) {
                    y0 = 0;
                    y1 = nc[k][1] - 1;
                }
                for (int b = y0; b <= y1; ++b) {
                    int bb = b;
                    if (P->periodic[1]) bb = ((b % nc[k][1]) + nc[k][1]) % nc[k][1];
                    else if (b < 0 || b >= nc[k][1]) continue;
                    for (int a = x0; a <= x1; ++a) {
                        int aa = a;
                        if (P->periodic[0]) aa = ((a % nc[k][0]) + nc[k][0]) % nc[k][0];
                        else if (a < 0 || a >= nc[k][0]) continue;
                        for (int j = head[k][(long long)bb * nc[k][0] + aa]; j >= 0;
                             j = next[j])
                            if (orc_is_neighbor(P, x[i], y[i], h[i], x[j], y[j], h[j])) {
                                if (pass == 1) nbr[kbase + c] = j;
                                ++c;
                            }
                    }
                }
            }
            if (pass == 0)
                cnt[i] = c;
            else
                qsort(nbr + kbase, (size_t)c, sizeof(int), cmp_int);
        }
    }
    long long tot = off[n];
    for (int k = 0; k < ncls; ++k) free(head[k]);
    free(cnt); free(next); free(bx); free(by); free(cls);
    return tot;
}

static int *g_boff = NULL, *g_bnbr = NULL;
static long long g_bcap = 0;
static int g_boffn = 0;

static void bg_neighbors(const orc_params *P, const orc_bgset *b) {
    int n = b->n;
    if (g_boffn < n + 1) {
        free(g_boff);
        g_boff = (int *)malloc((size_t)(n + 1) * sizeof(int));
        g_boffn = n + 1;
    }
    for (;;) {
        long long tot = orc_neighbors_classes(P, n, b->x, b->y, b->h, g_boff,
                                              g_bnbr, g_bcap);
        if (tot <= g_bcap) return;
        free(g_bnbr);
        g_bcap = tot + tot / 4 + 64;
        g_bnbr = (int *)malloc((size_t)g_bcap * sizeof(int));
    }
}

int orc_bg_iterations(const orc_bg_params *B) {
    return 3 * (int)ceil(log(B->ds_max / B->ds_min) / log(B->Cr));
}

/* Vorticity of the fluid, omega = dv/dx - du/dy, with the gradient operator
 * of the Taylor correction: omega_i = sum_{j != i} V_j ((v_j - v_i) dW/dx -
 * (u_j - u_i) dW/dy), grad W = grad_i W(r_ij, h_i), V_j = m_j / rho_j (the
 * paper names vorticity as its adaptivity measure without an operator). */
void orc_vorticity(const orc_params *P, const orc_state *s, double *omega) {
    int n = s->n;
    neighbors_auto(P, n, s->x, s->y, s->h);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double w = 0.0;
        for (int k = g_off[i]; k < g_off[i + 1]; ++k) {
            int j = g_nbr[k];
            if (j == i) continue;
            double dx, dy;
            separation(P, s->x[i], s->y[i], s->x[j], s->y[j], &dx, &dy);
            double r = sqrt(dx * dx + dy * dy);
            if (!(r > 0.0)) continue;
            double g = orc_dWdr(r, s->h[i]) / r;
            double Vj = s->m[j] / s->rho[j];
            w += Vj * ((s->v[j] - s->v[i]) * (g * dx) - (s->u[j] - s->u[i]) * (g * dy));
        }
        omega[i] = w;
    }
}

/* Step 1.  mark[b] = 1: a solid particle in range; 2: otherwise phi_b >
 * vort_k max|omega| (when vort_k > 0 and phi is given: phi_f = |omega_f| of
 * fluid particle f, phi_b the largest phi_f over fluid particles in range);
 * 0: neither.  Marked particles take ds = ds_min.  Returns the marked count. */
int orc_bg_mark(const orc_params *P, const orc_bg_params *B, orc_bgset *b,
                int nw, const double *wx, const double *wy, const double *wh,
                int nf, const double *fx, const double *fy, const double *fh,
                const double *phi, unsigned char *mark) {
    double pmax = 0.0;
    int use_phi = B->vort_k > 0.0 && nf > 0 && phi;
    if (use_phi)
        for (int f = 0; f < nf; ++f)
            if (phi[f] > pmax) pmax = phi[f];
    double thr = B->vort_k * pmax;
    int count = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : count)
    for (int i = 0; i < b->n; ++i) {
        unsigned char mk = 0;
        for (int s = 0; s < nw && !mk; ++s)
            if (orc_is_neighbor(P, b->x[i], b->y[i], b->h[i], wx[s], wy[s], wh[s]))
                mk = 1;
        if (!mk && use_phi && pmax > 0.0) {
            double pb = 0.0;
            for (int f = 0; f < nf; ++f)
                if (orc_is_neighbor(P, b->x[i], b->y[i], b->h[i], fx[f], fy[f], fh[f]) &&
                    phi[f] > pb)
                    pb = phi[f];
            if (pb > thr) mk = 2;
        }
        mark[i] = mk;
        if (mk) {
            b->ds[i] = B->ds_min;
            ++count;
        }
    }
    return count;
}

/* Step 2 (Jacobi over the unmarked particles). */
void orc_bg_size(const orc_params *P, const orc_bg_params *B, orc_bgset *b,
                 const unsigned char *mark) {
    int n = b->n;
    bg_neighbors(P, b);
    double *nds = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    const double cr3 = B->Cr * B->Cr * B->Cr;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        if (mark[i]) {
            nds[i] = b->ds[i];
            continue;
        }
        double lo = DBL_MAX, hi = 0.0, slog = 0.0;
        int c = 0;
        for (int k = g_boff[i]; k < g_boff[i + 1]; ++k) {
            int j = g_bnbr[k];
            if (j == i) continue;
            double s = b->ds[j];
            if (s < lo) lo = s;
            if (s > hi) hi = s;
            slog += log(s);
            ++c;
        }
        double d = b->ds[i];
        if (c > 0) d = (hi / lo < cr3) ? B->Cr * lo : exp(slog / c);
        if (d > B->ds_max) d = B->ds_max;
        if (d < B->ds_min) d = B->ds_min;
        nds[i] = d;
    }
    memcpy(b->ds, nds, sizeof(double) * (size_t)n);
    free(nds);
}

/* Step 3: parents are the particles with m > 1.05 rho0 ds^2; children as
 * in orc_split (ring at eps h, angles k pi/3, h = alpha h, m / 7, centre
 * keeps the id, ring ids next_id + 6 r + k with r the parent's rank in id
 * order) and copy ds.  Returns the parents, or -1 over capacity. */
int orc_bg_split(const orc_params *P, orc_bgset *b, long long *next_id) {
    int n = b->n;
    id_idx *par = (id_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(id_idx));
    int np = 0;
    for (int i = 0; i < n; ++i) {
        double mref = P->rho0 * b->ds[i] * b->ds[i];
        if (b->m[i] > 1.05 * mref) {
            par[np].id = b->id[i];
            par[np].idx = i;
            ++np;
        }
    }
    if ((long long)n + 6LL * np > b->cap) {
        free(par);
        return -1;
    }
    qsort(par, (size_t)np, sizeof(id_idx), cmp_id_idx);
    for (int r = 0; r < np; ++r) {
        int i = par[r].idx;
        double m = b->m[i], h = b->h[i];
        double mc = m / 7.0;
        double rad = P->split_eps * h;
        for (int k = 0; k < 6; ++k) {
            int c = n + 6 * r + k;
            b->x[c] = wrap(P, 0, b->x[i] + rad * HEX_C[k]);
            b->y[c] = wrap(P, 1, b->y[i] + rad * HEX_S[k]);
            b->m[c] = mc;
            b->h[c] = P->split_alpha * h;
            b->ds[c] = b->ds[i];
            b->id[c] = *next_id + 6LL * r + k;
        }
        b->m[i] = m - 6.0 * mc;
        b->h[i] = P->split_alpha * h;
    }
    b->n = n + 6 * np;
    *next_id += 6LL * np;
    free(par);
    return np;
}

/* Eq. h-smoothing (Jacobi): h_i <- (1/2) ((h_i/2)(1 + sqrt(N_r / N_i)) +
 * sum_j h_j / N_i) over the background N(i), i included. */
void orc_bg_hsmooth(const orc_params *P, const orc_bg_params *B, orc_bgset *b) {
    int n = b->n;
    bg_neighbors(P, b);
    double *nh = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double sh = 0.0;
        int c = 0;
        for (int k = g_boff[i]; k < g_boff[i + 1]; ++k) {
            sh += b->h[g_bnbr[k]];
            ++c;
        }
        double Ni = (double)c;
        nh[i] = 0.5 * (0.5 * b->h[i] * (1.0 + sqrt(B->Nr / Ni)) + sh / Ni);
    }
    memcpy(b->h, nh, sizeof(double) * (size_t)n);
    free(nh);
}

/* One shifting step of the background alone: Eqs. shift-deltar and
 * shift-limit with the readings of pass A (h_ij = mean h, denominator the
 * kernel at its inflection point, volume m_j / rho0). */
void orc_bg_shift(const orc_params *P, orc_bgset *b) {
    const double w_xi = w_of_q(XI_INFLECTION);
    int n = b->n;
    bg_neighbors(P, b);
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * 2 * sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        double ax = 0.0, ay = 0.0;
        for (int k = g_boff[i]; k < g_boff[i + 1]; ++k) {
            int j = g_bnbr[k];
            if (j == i) continue;
            double dx, dy;
            separation(P, b->x[i], b->y[i], b->x[j], b->y[j], &dx, &dy);
            double r = sqrt(dx * dx + dy * dy);
            if (!(r > 0.0)) continue;
            double hb = 0.5 * (b->h[i] + b->h[j]);
            double ratio = w_of_q(r / hb) / w_xi;
            double f = (b->m[j] / P->rho0) * (1.0 + 0.24 * p4(ratio)) *
                       orc_dWdr(r, hb) / r;
            ax += f * dx;
            ay += f * dy;
        }
        double c = -0.5 * b->h[i] * b->h[i];
        double sx = c * ax, sy = c * ay;
        double mag = sqrt(sx * sx + sy * sy);
        double lim = 0.25 * b->h[i];
        if (mag > lim) {
            double th = lim / mag;
            sx *= th;
            sy *= th;
        }
        d[2 * i] = sx;
        d[2 * i + 1] = sy;
    }
    for (int i = 0; i < n; ++i) {
        b->x[i] = wrap(P, 0, b->x[i] + d[2 * i]);
        b->y[i] = wrap(P, 1, b->y[i] + d[2 * i + 1]);
    }
    free(d);
}

int orc_bg_iteration(const orc_params *P, const orc_bg_params *B,
                     orc_bgset *b, long long *next_id, int nw,
                     const double *wx, const double *wy, const double *wh,
                     int nf, const double *fx, const double *fy,
                     const double *fh, const double *phi, orc_bg_stats *st) {
    orc_bg_stats z;
    memset(&z, 0, sizeof(z));
    z.n_before = b->n;
    unsigned char *mark = (unsigned char *)malloc((size_t)(b->n > 0 ? b->n : 1));
    z.n_marked = orc_bg_mark(P, B, b, nw, wx, wy, wh, nf, fx, fy, fh, phi, mark);
    for (int i = 0; i < b->n; ++i) z.n_vort += mark[i] == 2;
    orc_bg_size(P, B, b, mark);
    free(mark);
    int ns = orc_bg_split(P, b, next_id);
    if (ns < 0) {
        if (st) *st = z;
        return -1;
    }
    z.n_split = ns;
    for (int r = 0; r < B->smooth_iters; ++r) {
        orc_bg_hsmooth(P, B, b);
        orc_bg_shift(P, b);
    }
    z.n_after = b->n;
    if (st) *st = z;
    return 0;
}
