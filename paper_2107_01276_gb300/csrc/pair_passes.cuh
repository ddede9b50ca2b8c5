// Argument blocks and launchers of the pair passes, PEC stages and
// time-step reduction (pair_passes.cu).
#pragma once

#include "batch.cuh"
#include "kernels.cuh"
#include "neighbors.cuh"
#include "sph_internal.cuh"
#include "walls.cuh"

namespace sph {

template <typename R>
struct PassAArgs {
    int n;
    Domain d;
    Anchor an;
    const uint32_t *off, *list;  // CSR neighbour lists
    const float4 *pk;          // anchor coordinates (mixed path)
    const double *x, *y, *h;   // FP64 positions and smoothing lengths
    const R *m, *p, *u, *v;    // pair-arithmetic copies
    WallView w;
    double rho0;
    R *rho, *beta, *pavg, *drx, *dry, *V, *rb2;
    int *nnb;
    // per-particle records for pass B: {m, V, rho, 1/(rho^2 beta)} and
    // {p, u, v, 1/h}
    typename V4<R>::T *nbA, *nbB;
    int filter;                // 1: lists with a skin, test membership
};

template <typename R>
struct PassBArgs {
    int n;
    Domain d;
    Anchor an;
    const uint32_t *off, *list;
    const float4 *pk;
    const double *x, *y, *h;
    const R *m, *p, *u, *v;
    WallView w;
    const R *rho, *beta, *pavg, *drx, *dry, *V, *rb2;
    const typename V4<R>::T *nbA, *nbB;
    const double *dt;          // device {dt, 1 / dt}
    double rho0, cs, nu, alpha_e;
    int pavg_mode, diff_denominator, rho_factor;
    R *dpdt, *dudt, *dvdt;
    int *nonfinite;
    int filter;                // 1: lists with a skin, test membership
};

template <typename R>
struct PecArgs {
    int n;
    Domain d;
    double f;                  // 0.5 predict, 1.0 correct
    int save;                  // 1: the current x, y, u, v, p are the stage
                               // start; copy them into x0..p0 first
    // with skin_err: a particle moving more than disp_lim h in this stage
    // sets *skin_err (the neighbour lists of the step no longer hold N(i))
    const double *h;
    double disp_lim;
    int *skin_err;
    const double *dt;          // device {dt, 1 / dt}
    // sponge layer (sph_params.sponge_width; corrector only): width (0:
    // off), its downstream edge, the target speed
    double sponge_w, sponge_x1, sponge_U;
    const double *x0, *y0, *u0, *v0, *p0;
    const R *dudt, *dvdt, *dpdt, *drx, *dry;
    double *x, *y, *u, *v, *p;
};

struct ConvList {
    const double *src[8];
    float *dst[8];
    int k;
};

// Force on the walls (Eq. force-sph, pressures without the average
// offset): per wall particle (sorted wall order) {f_p,x, f_p,y, f_visc,x,
// f_visc,y} into fw[4 k ..]; fluid rho, beta from pass A (type R).
template <typename R>
struct ForceArgs {
    WallView w;
    Grid g;                       // fluid cell structure (fresh)
    Domain d;
    Anchor an;
    const float4 *pk;             // fluid anchor data
    const double *x, *y, *h, *m, *u, *v, *p;
    const R *rho, *beta;
    double rho0, nu;
    double *fw;
};

// team: lanes per particle (1, 4, 16 or 32), anything else: by set size.
template <typename R> void launch_pass_a(cudaStream_t s, const PassAArgs<R> &a,
                                         int team = 0);
template <typename R> void launch_forces(cudaStream_t s, const ForceArgs<R> &a);
// Deterministic sum of the per-wall forces into total[4] and their copy in
// load order (id: load index of each sorted wall) into out[4 id ..].
void launch_forces_total(cudaStream_t s, int nw, const double *fw,
                         const int64_t *id, double *out, double *total);
template <typename R> void launch_pass_b(cudaStream_t s, const PassBArgs<R> &a,
                                         int team = 0);
template <typename R> void launch_pec(cudaStream_t s, const PecArgs<R> &a);
// batched phases: one persistent launch over the work items of several
// instances (team: threads per particle, 1, 4, 16 or 32)
template <typename R>
void launch_pass_a_batch(cudaStream_t s, int team, const PassAArgs<R> *args,
                         const BatchSpan &sp);
template <typename R>
void launch_pass_b_batch(cudaStream_t s, int team, const PassBArgs<R> *args,
                         const BatchSpan &sp);
void launch_wall_bc_batch(cudaStream_t s, int team, const WallBcArgs *args,
                          const BatchSpan &sp);
template <typename R>
void launch_pec_batch(cudaStream_t s, const PecArgs<R> *args, const BatchSpan &sp);
void launch_rho_store_batch(cudaStream_t s, const RhoStoreArgs *args, const BatchSpan &sp);
void launch_nbr_ids(cudaStream_t s, int n, const uint32_t *off,
                    const uint32_t *list, const int64_t *id, int64_t *out);
// Returns the number of kernels launched.
// h_min and the time step of several small sets (n <= dt_small_max()), one
// block each (batched step).
struct DtSmallRec {
    int n;
    const double *h;
    double U, cs, nu;
    unsigned long long *hmin_bits;
    double *dt, *tacc;
    int nsteps;
};
void launch_dt_small_batch(cudaStream_t s, const DtSmallRec *args, const BatchSpan &sp);
int dt_small_max();
int launch_dt(cudaStream_t s, int n, const double *h,
               unsigned long long *hmin_bits, double U, double cs, double nu,
               double *dt, double *tacc, int nsteps);
void launch_reset_bbox(cudaStream_t s, int *bbox, uint32_t *level_mask);
void launch_to_float(cudaStream_t s, int n, const ConvList &c);
void launch_float_to_double(cudaStream_t s, int n, const float *src,
                            double *dst);

}  // namespace sph
