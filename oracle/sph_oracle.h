/*
 * Plain FP64 CPU oracle for the adaptive-resolution weakly-compressible SPH
 * method of Muta & Ramachandran, "Efficient and Accurate Adaptive Resolution
 * for Weakly-Compressible SPH" (arXiv 2107.01276).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is
 * never part of it.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load it.  It shares no code, header,
 * constant table or helper with the CUDA library.
 *
 * Every routine is a direct transcription of the paper's equations in the
 * paper's order, in double precision, compiled with FMA contraction off.
 * Where the paper is silent or ambiguous the reading taken is stated next to
 * the routine that implements it.
 *
 * Arrays are caller-owned host arrays.  Particle i of a set is element i of
 * every array; "id" is the persistent particle identity.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double lo[2], hi[2];     /* domain box */
    int periodic[2];         /* 1: periodic along that axis (minimum image) */
    double rho0;             /* reference density */
    double cs;               /* artificial speed of sound */
    double nu;               /* kinematic viscosity */
    double U_ref;            /* reference speed U in the time-step rule */
    double hdx;              /* C in h = C (m/rho)^(1/d) */
    double alpha_e;          /* EDAC viscosity factor, 1.5 in the paper */
    double split_alpha;      /* child h factor, 0.9 */
    double split_eps;        /* child ring radius factor, 0.4 */
    int pavg_mode;           /* 0: p_avg,i subtracted from p_i and p_j; 1: literal p_avg,j for P_j */
    int edac_diff_denominator; /* 1: pressure-diffusion term divided by r^2 + eta */
    int edac_rho_factor;     /* 1: third EDAC sum multiplied by rho_i */
    int merge_iters;         /* merge rounds after a split pass (3) */
    int shift_iters;         /* shift + Taylor-correction rounds (3) */
} orc_params;

/* Fluid particle set with capacity; n changes under split/merge. */
typedef struct {
    int n, cap;
    double *x, *y, *u, *v, *p, *rho, *m, *h, *mmin, *mmax;
    long long *id;
} orc_state;

/* Per-particle outputs of one right-hand-side evaluation, with the
 * condition scales S_i = sum of |terms| used by the parity norm. */
typedef struct {
    double *rho, *beta, *pavg, *drx, *dry, *dpdt, *dudt, *dvdt;
    int *nnb;
    double *s_rho, *s_beta, *s_pavg, *s_drx, *s_dry, *s_dpdt, *s_dudt, *s_dvdt;
} orc_rhs_out;

/* ---- kernel (section 2, Eq. kernel) ---- */
double orc_W(double r, double h);
double orc_dWdr(double r, double h);

/* ---- neighbour predicate and searches (section 2, gather sums) ---- */
int orc_is_neighbor(const orc_params *P, double xi, double yi, double hi,
                    double xj, double yj, double hj);
/* CSR of N(i), each list ascending in j, i itself included.  Returns the
 * total entry count; if it exceeds cap only off[] is valid. */
long long orc_neighbors_brute(const orc_params *P, int n, const double *x,
                              const double *y, const double *h, int *off,
                              int *nbr, long long cap);
long long orc_neighbors_grid(const orc_params *P, int n, const double *x,
                             const double *y, const double *h, int *off,
                             int *nbr, long long cap);
/* Cross-set search: for each a in set A, the members b of set B with
 * r_ab < 3 max(h_a, h_b).  Brute force. */
long long orc_neighbors_cross(const orc_params *P, int na, const double *xa,
                              const double *ya, const double *ha, int nb,
                              const double *xb, const double *yb,
                              const double *hb, int *off, int *nbr,
                              long long cap);

/* ---- multi-level cell keys ---- */
int orc_max_level(const orc_params *P, double c0);
void orc_cell_keys(const orc_params *P, double c0, int n, const double *x,
                   const double *y, const double *h, uint64_t *key,
                   int *level);

/* ---- right-hand side ---- */
int orc_pass_a(const orc_params *P, int n, const double *x, const double *y,
               const double *h, const double *m, const double *p,
               const int *off, const int *nbr, orc_rhs_out *o);
void orc_pass_b(const orc_params *P, double dt, int n, const double *x,
                const double *y, const double *h, const double *m,
                const double *p, const double *u, const double *v,
                const int *off, const int *nbr, orc_rhs_out *o);
double orc_dt(const orc_params *P, int n, const double *h);
/* Neighbour search + pass A + pass B at the current state. */
int orc_rhs(const orc_params *P, double dt, const orc_state *s,
            orc_rhs_out *o);
/* nsteps PEC steps; *t advanced by the sum of the time steps. */
int orc_step(const orc_params *P, orc_state *s, int nsteps, double *t);
/* The PEC stage updates alone, for tests with prescribed rates. */
void orc_pec_predict(const orc_params *P, double dt, int n, const double *x0,
                     const double *y0, const double *u0, const double *v0,
                     const double *p0, const double *dudt,
                     const double *dvdt, const double *dpdt,
                     const double *drx, const double *dry, double *x,
                     double *y, double *u, double *v, double *p);
void orc_pec_correct(const orc_params *P, double dt, int n, const double *x0,
                     const double *y0, const double *u0, const double *v0,
                     const double *p0, const double *dudt,
                     const double *dvdt, const double *dpdt,
                     const double *drx, const double *dry, double *x,
                     double *y, double *u, double *v, double *p);

/* ---- dummy wall particles (section 2.2) ---- */
/* Register the wall set used by orc_rhs / orc_step (copied; n = 0 clears
 * it): positions, smoothing lengths, masses and prescribed velocities. */
void orc_set_walls(int n, const double *x, const double *y, const double *h,
                   const double *m, const double *uw, const double *vw);
/* Wall pressure and extrapolated velocity from the fluid (Eqs. bc-wall,
 * shepard, bc-pre with g = a_w = 0) for the registered walls. */
/* Force on the solid (walls) at the state: {f_p,x, f_p,y, f_visc,x,
 * f_visc,y} (section "Force computation", Eq. force-sph, reading F1). */
void orc_forces(const orc_params *P, const orc_state *s, double *out,
                double *per_wall);
/* Test instrumentation: when acc (4 doubles per fluid particle) is set,
 * pass B writes each particle's wall terms of its momentum rate there
 * (pressure x, y, viscous x, y); NULL stops it. */
void orc_record_wall_terms(double *acc);
/* The wall condition at the state, kept for the registered walls (what
 * orc_rhs does first; for callers of orc_pass_a / orc_pass_b). */
void orc_wall_bc_store(const orc_params *P, const orc_state *s);
void orc_wall_bc(const orc_params *P, const orc_state *s, double *pw,
                 double *ugx, double *ugy);

/* ---- adaptive refinement (section 3) ---- */
typedef struct {
    long long n_before, n_split, n_merged, n_after;
    double mass_before, mass_after;
} orc_adapt_stats;

/* Fluid m_ref from background particles (section 3.3): m_min, m_max. */
void orc_bg_resolution(const orc_params *P, orc_state *s, int nb,
                       const double *bx, const double *by, const double *bh,
                       const double *bds);
/* One split pass (section 3.1); returns the number of parents split, or
 * -1 if the children would exceed the capacity (state unchanged). */
int orc_split(const orc_params *P, orc_state *s, long long *next_id);
/* One parallel mutual-closest merge round (section 3.2); returns pairs. */
int orc_merge_round(const orc_params *P, orc_state *s);
/* Shift displacement and Taylor gradients at the current state (no
 * update); g* hold the x and y components of grad u, grad v, grad p. */
void orc_shift_compute(const orc_params *P, const orc_state *s, double *rho,
                       double *drx, double *dry, double *gux, double *guy,
                       double *gvx, double *gvy, double *gpx, double *gpy);
/* One shift round: shift by dr and Taylor-correct u, v, p (Eqs. shift,
 * shift-correct). */
void orc_shift_round(const orc_params *P, orc_state *s);
/* Smoothing length from the neighbourhood-average mass (section 3.1). */
void orc_h_update(const orc_params *P, orc_state *s);
/* The whole adaptation of one iteration (section 3.4, ii-iii). */
int orc_adapt(const orc_params *P, orc_state *s, int nb, const double *bx,
              const double *by, const double *bh, const double *bds,
              long long *next_id, orc_adapt_stats *st);

/* ---- background particles (section 3.3) ---- */
typedef struct {
    int n, cap;
    double *x, *y, *h, *m, *ds;   /* ds: particle size, m_ref = rho0 ds^2 */
    long long *id;
} orc_bgset;
typedef struct {
    double ds_min, ds_max;   /* finest and coarsest size */
    double Cr;               /* size ratio of adjacent layers */
    double Nr;               /* reference neighbour count, Eq. h-smoothing (48) */
    int smooth_iters;        /* h-smoothing + shifting repetitions (3) */
    double vort_k;           /* > 0: vorticity marking threshold factor */
} orc_bg_params;
typedef struct {
    long long n_before, n_marked, n_vort, n_split, n_after;
} orc_bg_stats;
/* Same sets as orc_neighbors_brute, for sets whose h spans a wide range. */
long long orc_neighbors_classes(const orc_params *P, int n, const double *x,
                                const double *y, const double *h, int *off,
                                int *nbr, long long cap);
/* 3 ceil(log(ds_max / ds_min) / log Cr). */
int orc_bg_iterations(const orc_bg_params *B);
/* omega_i = sum_{j != i} V_j ((v_j - v_i) dW/dx - (u_j - u_i) dW/dy). */
void orc_vorticity(const orc_params *P, const orc_state *s, double *omega);
/* The steps of one construction iteration, and the iteration itself
 * (phi: |omega| of the nf fluid particles, or NULL). */
int orc_bg_mark(const orc_params *P, const orc_bg_params *B, orc_bgset *b,
                int nw, const double *wx, const double *wy, const double *wh,
                int nf, const double *fx, const double *fy, const double *fh,
                const double *phi, unsigned char *mark);
void orc_bg_size(const orc_params *P, const orc_bg_params *B, orc_bgset *b,
                 const unsigned char *mark);
int orc_bg_split(const orc_params *P, orc_bgset *b, long long *next_id);
void orc_bg_hsmooth(const orc_params *P, const orc_bg_params *B, orc_bgset *b);
void orc_bg_shift(const orc_params *P, orc_bgset *b);
int orc_bg_iteration(const orc_params *P, const orc_bg_params *B,
                     orc_bgset *b, long long *next_id, int nw,
                     const double *wx, const double *wy, const double *wh,
                     int nf, const double *fx, const double *fy,
                     const double *fh, const double *phi, orc_bg_stats *st);
int orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
