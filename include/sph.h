/*
 * sph.h -- C ABI of the GB300-native adaptive-resolution weakly-compressible
 * SPH library (Muta & Ramachandran, "Efficient and Accurate Adaptive
 * Resolution for Weakly-Compressible SPH", arXiv 2107.01276).
 *
 * The library advances one 2-D particle simulation per context on one GPU.
 * Every numerical step runs in the library's own CUDA kernels (sm_103a);
 * there is no CPU fallback.  Paper references are to its sections and its
 * equation labels.
 *
 * Conventions
 *  - Ownership: the library allocates and owns all device memory of a
 *    context (sized by sph_params.capacity at sph_create).  Callers own
 *    every host buffer they pass; every transfer is a copy.
 *  - Streams: all device work of a context is enqueued on the stream given
 *    to sph_create (a cudaStream_t; NULL = the legacy default stream).
 *    sph_load_particles, sph_rhs, sph_step and sph_adapt return once their
 *    work is enqueued, except where stated; sph_read synchronises.
 *  - Errors: every call returns an sph_status and never throws or aborts.
 *    After any status other than SPH_ECUDA the context stays usable;
 *    sph_last_error() gives a one-line message.  A NULL context gives
 *    SPH_EINVAL.
 *  - Particle order: the library keeps particles sorted by cell key and
 *    re-sorts them whenever it rebuilds the neighbour structure.  sph_read
 *    returns every field of one state in the same (current) order;
 *    SPH_F_ID gives each particle's persistent identity.
 *  - Precision: SPH_FP64 computes everything in double.  SPH_MIXED keeps
 *    positions, time integration, masses, split/merge bookkeeping and the
 *    time-step reduction in double and does the pair arithmetic of the
 *    right-hand side in float with float accumulation.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_EINVAL = 1,      /* bad argument; nothing was changed */
    SPH_ENOMEM = 2,      /* device allocation failed */
    SPH_ECUDA = 3,       /* CUDA runtime error; the context must be destroyed */
    SPH_ECAPACITY = 4,   /* particle count would exceed sph_params.capacity */
    SPH_ENONFINITE = 5,  /* a rate or state value became NaN/Inf */
    SPH_ETIMEOUT = 6,    /* a bounded device wait gave up */
    SPH_ESTATE = 7       /* call not valid in the current state (e.g. no fluid loaded) */
} sph_status;

typedef enum {
    SPH_FLUID = 0,
    SPH_WALL = 1,
    SPH_BACKGROUND = 2,
    SPH_REGION = 3   /* markers of a user-specified refinement region */
} sph_kind;
typedef enum { SPH_FP64 = 0, SPH_MIXED = 1 } sph_precision;

/* Problem parameters (SI units).  sph_default_params fills the paper's
 * values; the reading switches take the defaults stated beside them. */
typedef struct {
    int dim;                 /* must be 2 (the paper is two-dimensional) */
    double lo[2], hi[2];     /* domain box; positions stay in it */
    int periodic[2];         /* 1: periodic axis, minimum-image pairs */
    double rho0;             /* reference density */
    double cs;               /* artificial speed of sound (section 2) */
    double nu;               /* kinematic viscosity */
    double U_ref;            /* speed U of the time-step rule (section 2.4) */
    double hdx;              /* C of h = C (m/rho)^(1/d) (section 3.1) */
    double alpha_e;          /* EDAC viscosity factor, Eq. edac-alpha: 1.5 */
    double split_alpha;      /* child smoothing-length factor (section 3.1): 0.9 */
    double split_eps;        /* child ring radius / h (section 3.1): 0.4 */
    double Cr;               /* layer size ratio (section 3.3): 1.08 */
    double ds_min, ds_max;   /* finest / coarsest particle spacing (section 3.3) */
    int merge_iters;         /* merge rounds after splitting (section 3.2): 3 */
    int shift_iters;         /* shift + Taylor rounds (section 3.2): 3 */
    int precision;           /* sph_precision */
    long long capacity;      /* maximum fluid particles held on the device */
    int pavg_mode;           /* 0 (default): P_j = (p_j - p_avg,i)/(rho_j^2 beta_j);
                                1: literal Eq. mom:pre with p_avg,j */
    int edac_diff_denominator; /* 1 (default): EDAC diffusion sum divided by r^2+eta */
    int edac_rho_factor;     /* 1 (default): third EDAC sum multiplied by rho_i */
    double cell_c0;          /* level-0 cell side of the neighbour grid;
                                <= 0: 3*hdx*ds_min if ds_min > 0, else 3*min(h)
                                of the fluid at load time */
    /* background construction (section 3.3, sph_background) */
    double bg_Nr;            /* reference neighbour count N_r of Eq.
                                h-smoothing: 48 */
    int bg_smooth_iters;     /* h-smoothing + shifting repetitions per
                                iteration: 3 */
    double vort_k;           /* > 0: solution adaptivity, background particles
                                near fluid with |omega| > vort_k max|omega|
                                take ds_min (0.05 in the paper's runs);
                                <= 0 (default): off */
    int n_bg;                /* > 0: every n_bg-th sph_adapt call first runs
                                one background iteration; 0 (default): never */
    long long bg_capacity;   /* maximum background particles during the
                                construction; <= 0: max(100 x the loaded
                                count, 2^18) */
    double sponge_width;     /* > 0: a sponge layer of this width at the low-x
                                end of the box (flow along +x) relaxes u ->
                                U_ref, v -> 0, p -> 0 at the end of each PEC
                                step, by the fraction min(1, 10 U_ref dt / w
                                s^2), s = 1 at the low-x edge falling to 0 at
                                its downstream edge; the periodic cylinder
                                stand-in's inflow (the paper's inlet and
                                outlet are not defined in it).  0
                                (default): off */
} sph_params;

/* Host arrays of one particle set, n entries each.  Unused members may be
 * NULL: u, v, p, rho default to 0, 0, 0, rho0; id defaults to 0..n-1 and
 * ds (background only) to ds_max; mmin/mmax default to 0. */
typedef struct {
    const double *x, *y, *u, *v, *p, *rho, *m, *h;
    const double *mmin, *mmax, *ds;
    const int64_t *id;
} sph_particles;

/* Fields sph_read can copy out.  Doubles unless noted. */
typedef enum {
    SPH_F_X = 0, SPH_F_Y, SPH_F_U, SPH_F_V, SPH_F_P, SPH_F_RHO, SPH_F_M,
    SPH_F_H, SPH_F_MMIN, SPH_F_MMAX,
    SPH_F_ID,          /* int64 */
    SPH_F_BETA, SPH_F_PAVG, SPH_F_DRX, SPH_F_DRY,   /* last pass A */
    SPH_F_DPDT, SPH_F_DUDT, SPH_F_DVDT,             /* last pass B */
    SPH_F_NNB,         /* int32: |N(i)| of the last pass A, i included */
    /* The next three describe the current positions.  If particles moved
     * since the last rebuild, reading one rebuilds first, which re-sorts
     * the particles (read SPH_F_ID after them) and drops the last
     * right-hand side. */
    SPH_F_CELLKEY,     /* uint64: level << 58 | morton(ix, iy) */
    SPH_F_NEIGH_OFF,   /* int64[n+1]: CSR offsets of N(i) */
    SPH_F_NEIGH_ID,    /* int64[total]: ids of N(i), any order within a list */
    SPH_F_OMEGA,       /* vorticity of the fluid at the current positions
                          (rebuilds first like SPH_F_CELLKEY) */
    /* The background set (section 3.3), n_bg entries in the library's
     * order; SPH_F_BG_ID gives each particle's identity (load index, or
     * assigned by splitting during sph_background). */
    SPH_F_BG_X, SPH_F_BG_Y, SPH_F_BG_H, SPH_F_BG_M, SPH_F_BG_DS,
    SPH_F_BG_ID,       /* int64 */
    SPH_F_COUNT
} sph_field;

/* OR-ed into the field of sph_read: the fluid rows in ascending id order
 * instead of the library's current (cell-key) order, for comparing results
 * particle by particle.  Taken by the per-particle fields SPH_F_X ...
 * SPH_F_CELLKEY and SPH_F_OMEGA. */
#define SPH_READ_BY_ID 0x100

typedef struct {
    long long n;          /* fluid particles */
    long long n_wall;     /* wall (dummy) particles */
    long long n_bg;       /* background particles */
    double t;             /* simulated time advanced by sph_step */
    double dt;            /* time step of the last sph_step (Eq. timestep) */
    double c0;            /* level-0 cell side in use */
    int levels;           /* number of cell levels (top level spans the domain) */
    long long steps;      /* PEC steps taken */
    long long launches;   /* kernels launched by this context so far */
    long long next_id;    /* id the next split child will receive */
    long long n_region;   /* refinement-region markers */
    long long graph_steps; /* sph_step steps run as replayed CUDA graphs */
} sph_info;

/* Counts and masses of one sph_adapt call. */
typedef struct {
    long long n_before;   /* fluid particles before */
    long long n_split;    /* parents split (each became 7 particles) */
    long long n_merged;   /* particles removed by merging, over all rounds */
    long long n_after;    /* fluid particles after */
    double mass_before, mass_after;   /* total fluid mass (FP64 sums) */
    long long n_bg_nearest;   /* fluid particles with no background particle
                                 in range (took the nearest one's size) */
} sph_adapt_stats;

/* Counts of one sph_background call. */
typedef struct {
    long long n_before;   /* background particles before */
    long long n_marked;   /* last iteration: particles set to ds_min */
    long long n_vort;     /* ... of them by the vorticity criterion */
    long long n_split;    /* parents split, over all iterations */
    long long n_after;    /* background particles after */
    int iterations;       /* iterations run */
} sph_bg_stats;

typedef struct sph_ctx sph_ctx;

/* Fill *p with the paper's values: alpha_e 1.5, split_alpha 0.9,
 * split_eps 0.4, Cr 1.08, 3 merge and 3 shift rounds, hdx 1.0, and the
 * default readings; domain [0,1]^2 non-periodic, rho0 1, cs 10, nu 0,
 * U_ref 1, precision FP64, capacity 0 (must be set). */
void sph_default_params(sph_params *p);

/* Validate *p and allocate a context with device storage for
 * p->capacity fluid particles.  stream: cudaStream_t (may be NULL).  The
 * context's device buffers come from CUDA's stream-ordered allocator on
 * that stream (cudaMallocAsync / cudaFreeAsync): creating, growing and
 * destroying a context never synchronise the whole device.  The call
 * synchronises the stream before it returns.
 * Errors: SPH_EINVAL (dim != 2, empty box, capacity <= 0, non-positive
 * rho0/cs/hdx, negative nu), SPH_ENOMEM, SPH_ECUDA.  *out is NULL on error. */
sph_status sph_create(const sph_params *p, void *stream, sph_ctx **out);

/* Replace the particle set of the given kind by n particles copied from
 * host arrays.  SPH_FLUID: x, y, m, h required (see sph_particles for
 * defaults).  SPH_BACKGROUND (section 3.3): x, y, h required; ds (the
 * particle size; NULL takes ds_max), m (NULL: rho0 ds^2, used only by
 * sph_background) and id (NULL: 0..n-1) optional, any count; the set only
 * sets the fluid's m_min/m_max in sph_adapt and is refined by
 * sph_background.  SPH_WALL (section 2.2): x, y, h, m required, u, v the
 * prescribed wall velocity (NULL: 0); the walls also serve as the solid of
 * the background construction.  SPH_REGION (section 3.3, user-specified
 * regions): x, y, h of marker particles that act as a solid for the
 * background construction's boundary marking only; they take no part in
 * the flow.
 * Fluid positions must lie in the box (periodic axes: [lo, hi)).  A fluid
 * set is copied into the context's spare buffers and checked there on the
 * device (h and m positive and finite, positions finite and in the box,
 * the least and largest h, the largest id); only a set that passes
 * replaces the current one, so on SPH_EINVAL the context keeps its state.
 * Synchronous with respect to the host buffers (they may be reused on
 * return).  Errors: SPH_EINVAL (NULL required array, n < 0, h or m not
 * positive and finite, position outside the box), SPH_ECAPACITY
 * (n > capacity), SPH_ECUDA. */
sph_status sph_load_particles(sph_ctx *ctx, sph_kind kind, long long n,
                              const sph_particles *src);

/* One right-hand-side evaluation at the current state (section 2): rebuild
 * the cell structure, pass A (summation density Eq. sd-gather, beta Eq.
 * beta, p_avg Eq. pavg, limited shift Eqs. shift-deltar / shift-limit),
 * pass B (EDAC pressure rate Eq. edac:sph, momentum rate Eq. mom-sph),
 * with dt from Eq. timestep for u~ - u = dr/dt.  Results are read with
 * sph_read (SPH_F_RHO ... SPH_F_DVDT).  Errors: SPH_ESTATE (no fluid). */
sph_status sph_rhs(sph_ctx *ctx);

/* nsteps predict-evaluate-correct steps (section 2.4, Eqs. int-pre and
 * int-cor; two right-hand sides per step; dt from Eq. timestep).  If
 * t_out is not NULL it receives the simulated time after the steps, which
 * requires one synchronisation.  SPH_MIXED builds the neighbour lists once
 * per step with a skin (radius 1.1 x 3 max(h_i, h_j)); pass A tests
 * membership (N_i and p_avg count members only) and pass B's terms vanish
 * beyond the kernel support, so both evaluations see exactly N(i); a
 * particle that moves more than 0.15 h in the predictor invalidates that
 * and is reported (the time step and the shift limit keep moves below
 * 0.15 h for speeds up to 0.2 (U_ref + cs), i.e. Mach 0.2).  Errors:
 * SPH_ESTATE, SPH_EINVAL (nsteps < 0), SPH_ENONFINITE (a non-finite rate,
 * or a particle that outran the skin; checked at the end when t_out is
 * given, else at the next synchronising call; reported once: the state
 * then holds non-finite or invalid values, so load a state with
 * sph_load_particles before stepping on), SPH_ECAPACITY (neighbour-list
 * overflow, likewise). */
sph_status sph_step(sph_ctx *ctx, int nsteps, double *t_out);

/* Batched stepping: several independent simulations (of different sizes,
 * parameters and precisions, with or without walls) advance one PEC step
 * together.  A batch holds the device work lists of up to max_instances
 * contexts per call and the stream its launches go on (a cudaStream_t;
 * NULL = the legacy default stream); it owns no particle data.
 * sph_batch_create errors: SPH_EINVAL (out NULL, max_instances outside
 * 1 .. 2^20), SPH_ENOMEM.  sph_batch_destroy waits for the batch's work and
 * frees it (SPH_EINVAL for NULL). */
typedef struct sph_batch sph_batch;
sph_status sph_batch_create(int max_instances, void *stream, sph_batch **out);
sph_status sph_batch_destroy(sph_batch *batch);

/* One step of sph_step (nsteps = 1, section 2.4) for each of the k distinct
 * contexts ctx[0 .. k-1].  Each context's time step and neighbour build run
 * on its own stream; then every per-particle phase of the step (wall
 * conditions, pass A, pass B, the predictor and corrector stages, the
 * mid-step packing of SPH_MIXED contexts, the density store) runs on the
 * batch's stream as ONE persistent launch over all contexts that share a
 * precision and a team size, its work list made of (context, block of
 * particles) items.  The neighbour build of a context with at most 16384
 * particles, no wall lists and list sizes known from earlier builds runs
 * batched the same way (one launch per kernel of the build); other
 * contexts build on their own streams (SPH_FP64 contexts also mid-step).
 * Pass A / B thread-team sizes are those set by sph_set_tuning, else the
 * size rule applied to the batch's total particle count of that
 * precision; with the team sizes a context uses alone, its results equal
 * those of sph_step on it alone bit for bit (otherwise they differ by the
 * order of the pair sums).
 * The contexts' streams wait for the batch's launches before their next
 * work.  t_out (NULL or k entries) receives each context's simulated time
 * and makes the call synchronise and report the checks sph_step reports.
 * failed (may be NULL) receives the index of the context an error belongs
 * to, or -1; its sph_last_error() has the message.  Errors: SPH_EINVAL
 * (NULL batch, ctx or context, k outside 1 .. max_instances, a context
 * listed twice: nothing was changed), SPH_ESTATE (a context without fluid:
 * nothing was changed), and the errors of sph_step (a failed neighbour
 * build before the predictor leaves every context at its state before the
 * call; a failed mid-step build of an SPH_FP64 context leaves the batch
 * between the stages: reload the state). */
sph_status sph_batch_step(sph_batch *batch, sph_ctx *const *ctx, int k, double *t_out,
                          int *failed);

/* Kernel launches the batch itself issued so far (one per phase and group
 * and call; the contexts' own launches count in their sph_info). -1 for
 * NULL. */
long long sph_batch_launches(const sph_batch *batch);

/* Captured CUDA graphs of the batched step: once the same contexts (same
 * order, configuration and particle counts) have come up in three calls in
 * a row, the whole step -- every context's time step and build on its
 * stream and the batched phases -- is captured as one graph and replayed
 * while the batch recurs (two graphs alternate: each step swaps the
 * contexts' state buffers), with the same launches and results as the
 * launch-by-launch step.  Needs a batch stream other than the legacy or
 * per-thread default stream, library timing off on every context, and list
 * sizes known from earlier builds.  enable = 0 turns graphs off (default
 * on).  Errors: SPH_EINVAL (NULL batch).  sph_batch_graph_steps: steps
 * replayed as graphs so far (-1 for NULL). */
sph_status sph_batch_set_graphs(sph_batch *batch, int enable);
long long sph_batch_graph_steps(const sph_batch *batch);

/* One adaptation of the fluid particles (section 3, steps ii-iii of the
 * time loop in section 3.4), in FP64 for both precisions:
 *  1. if a background set is loaded, m_ref of each fluid particle is the
 *     smallest rho0 ds_b^2 over background particles b with r_ib <
 *     3 max(h_i, h_b), else that of the nearest one; m_max = 1.05 m_ref,
 *     m_min = 0.5 m_ref (section 3.3).  Without a background the loaded
 *     m_min/m_max stay; m_max <= 0 means no limit (never split or merged);
 *  2. one split pass: m > m_max -> 7 children (centre + hexagon at
 *     split_eps*h, h = split_alpha*h, mass m/7), children ids assigned from
 *     a counter in parent-id order (section 3.1);
 *  3. merge_iters rounds of mutual-closest merging (section 3.2,
 *     Eqs. merged-pos, merged-prop, merged-h);
 *  4. shift_iters rounds of limited shifting with Taylor correction of u,
 *     v, p (Eqs. shift, shift-deltar, shift-limit, shift-correct);
 *  5. h = hdx (mbar/rho)^(1/2) with the neighbourhood-average mass.
 * Synchronises (it reads back the particle counts).  out (may be NULL)
 * receives counts and total masses.  Errors: SPH_ESTATE (no fluid),
 * SPH_ECAPACITY (the children would exceed the capacity; nothing is split,
 * m_min/m_max are already refreshed). */
sph_status sph_adapt(sph_ctx *ctx, sph_adapt_stats *out);

/* sph_adapt for each of the k distinct contexts ctx[0 .. k-1].  The
 * contexts are shared out, in contiguous runs, over up to as many host
 * threads as the host has hardware threads (the caller's among them, each
 * on the caller's current device); each thread adapts its run in
 * lockstep: every phase of the adaptation (background construction when
 * due, split, each merge round, the shift rounds with the h update) is
 * issued for every context of the run still adapting, each on its own
 * context's stream, before one host synchronisation of all of them
 * gathers the counts the next phase needs (the split count, a merge
 * round's survivors, the masses).  So the contexts' kernels overlap on the
 * device, and a run of adaptations waits on about as many
 * synchronisations as one.  Each
 * context receives the kernels, in the order and with the arguments, of
 * sph_adapt on it alone: its state and stats equal sph_adapt's bit for
 * bit.  Nothing runs on the batch's stream; the next sph_batch_step orders
 * itself after the contexts' streams as always.  A context whose
 * adaptation fails stops where sph_adapt would stop (its message in its
 * sph_last_error) while the others go on.  stats: NULL or k entries
 * (zeroed for a failed context); status: NULL or k entries, each
 * context's own result.  Returns SPH_OK when every adaptation succeeded,
 * else the first failed context's status.  Errors before any work:
 * SPH_EINVAL (NULL batch, ctx or context, k outside 1 .. max_instances, a
 * context listed twice). */
sph_status sph_batch_adapt(sph_batch *batch, sph_ctx *const *ctx, int k,
                           sph_adapt_stats *stats, sph_status *status);

/* Background construction (section 3.3): `iterations` iterations over the
 * loaded background (iterations <= 0: 3 ceil(log(ds_max / ds_min) /
 * log Cr), the paper's count for the initial construction), each:
 *  1. a background particle with a wall or region-marker particle s in
 *     range (r_bs < 3 max(h_b, h_s)) takes ds_min; with vort_k > 0 and
 *     fluid loaded, so
 *     does one whose largest |omega| over fluid particles in range exceeds
 *     vort_k max|omega| (omega from the fluid's current state);
 *  2. every other particle takes, over its background neighbours j != i
 *     (same range rule, sizes after step 1, all read before any is
 *     written): Cr min_j ds_j if max_j ds_j / min_j ds_j < Cr^3, else the
 *     geometric mean of the ds_j; clamped to [ds_min, ds_max]; unchanged
 *     without neighbours;
 *  3. particles with m > 1.05 rho0 ds^2 split into seven as in sph_adapt
 *     (children copy ds; ids continue from the largest background id);
 *  4. bg_smooth_iters times: Eq. h-smoothing with N_r = bg_Nr over N(i)
 *     (i included), then one limited shifting step (Eqs. shift-deltar,
 *     shift-limit, volumes m_j / rho0) of the background alone.
 * Marking, sizes, splits and the h-smoothing in FP64; the shifting step's
 * pair sums in the context's precision (FP32 pair arithmetic over FP64
 * state for SPH_MIXED, as in sph_adapt).  The refined set replaces the loaded
 * background (read it with SPH_F_BG_*).  Synchronises (split counts).
 * out (may be NULL) receives counts.  Errors: SPH_ESTATE (no background),
 * SPH_EINVAL (ds_min, ds_max, Cr, bg_Nr not usable: need 0 < ds_min <=
 * ds_max, Cr > 1, bg_Nr > 0), SPH_ECAPACITY (the background would exceed
 * bg_capacity; the iterations before that are kept), SPH_ENOMEM. */
sph_status sph_background(sph_ctx *ctx, int iterations, sph_bg_stats *out);

/* Force on the solid, i.e. on the loaded wall particles, at the current
 * state (section "Force computation", Eq. force-sph): for each wall
 * particle w over its fluid neighbours j (r_wj < 3 max(h_w, h_j)),
 *   f_p,w    = -m_w sum_j m_j (P_w grad W(r_wj, h_w) + P_j grad W(r_wj, h_j))
 *   f_visc,w =  m_w / beta_w sum_j m_j 4 nu / (rho_w + rho_j)
 *                 (r_wj . grad W_wj) / (|r_wj|^2 + eta_w) (u_w - u_j)
 * with P_w = p_w / rho0^2 and P_j = p_j / (rho_j^2 beta_j) (pressures
 * without the average-pressure offset: a solid's sum sees fluid on one
 * side only, where the pressure level is the load), rho_w = rho0, beta_w
 * = 1, eta_w = 0.001 h_w^2, grad W_wj the mean of the two gradients and
 * u_w the wall's extrapolated velocity; p_w, u_w from the wall condition
 * and rho_j, beta_j from a pass A, all evaluated here at the current state
 * (a neighbour build and one right-hand side; the particle state is not
 * changed and the rates read afterwards are those of this state).  FP64
 * sums for both precisions.  total[4] = {f_p,x, f_p,y, f_visc,x,
 * f_visc,y}, summed over the walls in a fixed order; per_wall (may be
 * NULL) receives 4 doubles per wall particle in load order.  The drag and
 * lift coefficients of Eq. cdcl are these divided by rho0 U^2 L / 2.
 * Without walls every output is zero.  Synchronises.  Errors: SPH_EINVAL
 * (total NULL), SPH_ESTATE (no fluid), SPH_ENOMEM. */
sph_status sph_forces(sph_ctx *ctx, double *per_wall, double *total);

/* Drag and lift coefficients of the solid at the current state (section
 * "Force computation", Eq. cdcl): with the force of sph_forces and the
 * dynamic pressure q = rho0 U^2 L / 2 (U: free-stream speed, L:
 * characteristic length, e.g. the cylinder diameter), out[3] = {c_d
 * pressure = f_p,x / q, c_d skin friction = f_visc,x / q, c_l = f_p,y /
 * q}, the flow taken along +x.  Evaluates the state as sph_forces does.
 * Synchronises.  Errors: SPH_EINVAL (out NULL, U or L not positive), and
 * those of sph_forces. */
sph_status sph_force_coefficients(sph_ctx *ctx, double U, double L, double *out);

/* Launch configuration of a context's hot kernels.  Every choice gives the
 * same neighbour sets; the team sizes change the summation order of the
 * pair sums (results equal to rounding, not bit for bit). */
typedef struct {
    double cell_scale;   /* level-0 cell side = cell_scale x the default of
                            sph_params.cell_c0; <= 0: 1 */
    int walk;            /* list build: 1 per-particle team walk, 2 cell
                            tiles with 4-lane teams, 3 cell tiles with a
                            lane per particle, 4 the same with neighbouring
                            cells of a level merged into one chunk of at
                            most 32 particles (the same exact lists as 3);
                            0: by set size (< 12k: 1, < 48k: 2, else 4) */
    int team_a, team_b;  /* lanes per particle in pass A / pass B: 1, 4,
                            16 or 32; 0: by set size */
    int walls;           /* walls seen from the fluid: 1 the wall grid's
                            cells around each fluid particle, 2 wall lists
                            built with each neighbour build (from the walls'
                            side); 0: lists when there are at least 2048
                            wall particles */
    int no_graphs;       /* 0 (default): sph_step replays each step as a
                            captured CUDA graph when it can (the only live
                            context of the process, a stream other than the
                            legacy or per-thread default stream, timing
                            off, list sizes settled, two steps since the
                            particle set or configuration last changed);
                            results are the same bit for bit.  With several
                            contexts (the serving loop) capturing would wait
                            on the others' allocations and synchronisations,
                            so steps run launch by launch.  1: always launch
                            by launch */
    /* filled by sph_autotune: mean device ms per launch of each candidate
     * (neighbour build + both passes for cell_scale 1, 1.25, 1.5; the walk
     * for walk 1, 2, 4; pass A / pass B for teams 1, 4, 16, 32) */
    double ms_cell[3], ms_walk[3], ms_team_a[4], ms_team_b[4];
    double ms_walls[2];  /* build + both passes with walls 1, 2 (walls
                            loaded only) */
} sph_tune;

/* Autotuner (the paper has no counterpart; a launch-configuration search
 * for this GPU): on the loaded fluid set at its current state, times
 * neighbour builds and right-hand sides for each level-0 cell size
 * (x1, x1.25, x1.5), then each list-build kernel, then each team size of
 * pass A and pass B, then (with walls) the two ways the fluid sees the
 * walls (CUDA events, a few repetitions after a warm-up), and
 * keeps the fastest of each for this context; out (may be NULL) receives
 * the choices and the times.  It ends with a right-hand side as sph_rhs
 * does (the state re-sorted, its density the summation density, the rates
 * those of the current state); positions, velocities, pressures, masses
 * and h are not changed.  Takes a few dozen builds; clears the
 * sph_kernel_time accumulators; synchronises.  Errors: SPH_ESTATE (no fluid), others
 * as sph_rhs. */
sph_status sph_autotune(sph_ctx *ctx, sph_tune *out);

/* Sets a context's launch configuration (for instance one sph_autotune
 * found for another context of the same kind and size); the ms_* members
 * are ignored.  Errors: SPH_EINVAL (a value not listed above). */
sph_status sph_set_tuning(sph_ctx *ctx, const sph_tune *in);

/* Copy one field of the fluid set to the host buffer dst holding cap
 * elements of the field's type; *n_out (if not NULL) receives the element
 * count.  Rows come in the library's current order (read SPH_F_ID for the
 * identities), or by ascending id with SPH_READ_BY_ID.  Synchronises the
 * context's stream.  Errors: SPH_EINVAL (bad field, SPH_READ_BY_ID on a
 * field without per-particle rows, dst NULL), SPH_ECAPACITY (cap too
 * small; *n_out still set), SPH_ESTATE (field not computed yet). */
sph_status sph_read(sph_ctx *ctx, sph_field field, void *dst, long long cap,
                    long long *n_out);

/* Counts, time and time step of the context (synchronises). */
sph_status sph_get_info(sph_ctx *ctx, sph_info *out);

/* Kernel timing: when enabled the context records CUDA events around the
 * launches of each timed kernel family on its stream.  sph_kernel_time
 * returns the accumulated device milliseconds and launch count of one
 * family (0: pass B, 1: pass A, 2: neighbour rebuild (keys, sort, gather,
 * table, lists), 3: PEC stages, 4: adaptation (rebuilds inside it
 * included), 5: the neighbour walk of each rebuild alone, 6: the cell keys,
 * stable sort and gather of each rebuild alone) and resets them if reset
 * is non-zero.  Synchronises. */
sph_status sph_set_timing(sph_ctx *ctx, int enable);
sph_status sph_kernel_time(sph_ctx *ctx, int family, double *ms,
                           long long *launches, int reset);

/* Measured non-tensor FMA throughput of the current device (the paper has
 * no counterpart; the denominator of the pair passes' ALU rooflines, which
 * are plain FP32 / FP64 arithmetic).  Runs, on stream (a cudaStream_t; NULL
 * the legacy default stream), a few launches of a kernel in which every
 * thread of every SM's resident blocks advances 8 independent FMA chains
 * for ~20 ms, and returns the best rate in *flops (FLOP/s, an FMA counting
 * 2) and, if sms is not NULL, the multiprocessor count read from the
 * device.  fp64: 0 FP32, 1 FP64.  Allocates a few bytes; synchronises.
 * Errors: SPH_EINVAL (flops NULL, fp64 not 0/1), SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_probe_fma(int fp64, void *stream, double *flops, int *sms);

/* Debug builds (the library compiled with SPH_DEBUG; the paper has no
 * counterpart): the kernels check the indices of neighbour-list gathers,
 * the cell ranges of the list build, the sort's gather and the compaction
 * writes, and a failed check is counted and its access skipped (no trap,
 * no fault: the context stays usable).  sph_debug_failures returns the
 * failures counted since its last call on the current device (always 0 in
 * a release build) and synchronises; sph_debug_build returns 1 in a debug
 * build, else 0. */
unsigned long long sph_debug_failures(void);
int sph_debug_build(void);

/* Cell keys and stable sort of a particle set, allocating nothing.
 *
 * The paper has no counterpart to this entry point.  It serves callers
 * that cannot allocate device memory themselves: for example a solver
 * embedded in a host application that owns all device memory through its
 * own pool (a raw cudaMalloc/cudaFree would bypass that pool's accounting,
 * and cudaFree can stall the whole device), or a latency-critical loop
 * that must not pay for an allocation.  It computes, without a context,
 * the cell keys and stable order of the neighbour rebuild (the level of
 * each particle, then the Morton order of its cell).  They equal a
 * context's SPH_F_CELLKEY and SPH_F_ID order after sph_rhs when p->cell_c0
 * is that context's level-0 cell side (sph_get_info's c0, which includes
 * any sph_set_tuning / sph_autotune scale and, without ds_min, follows
 * from the smallest h loaded); the side used here has no tuning scale.
 * The scratch it needs is one
 * fixed device array inside the library, about 3.2 MB, reserved on every
 * GPU that loads the library until the process exits; the call itself
 * allocates nothing.
 *
 * x, y, h: device arrays of n particles (FP64).  key_out (uint64) and
 * perm_out (uint32): caller-owned device arrays of n entries, written with
 * the cell keys (level << 58 | morton(ix, iy)) in ascending order and, for
 * each sorted position, the input index of its particle (stable for equal
 * keys).  Level-0 cell side: p->cell_c0 if > 0, else 3 * p->hdx *
 * p->ds_min.  The work is enqueued on `stream` (cudaStream_t; NULL = the
 * legacy default stream) and the call returns once it is enqueued.
 *
 * Limits and sharing: n <= 262144 (SPH_EINVAL beyond).  Every call looks
 * up the fixed array's address on the current device (so a device reset
 * between calls is harmless); the first lookup on a device loads the
 * library's module there, so make the first call before any stream
 * capture.  Every call on a device uses the same array and each call
 * resets the parts it relies on, so calls whose work overlaps on the GPU
 * (different streams or host threads) race and must be serialised by the
 * caller.
 * Errors: SPH_EINVAL (NULL argument, n out of range, no cell side, bad
 * domain), SPH_ECUDA (device address lookup or launch failure); the reason
 * is then sph_last_error(NULL) on the calling thread. */
sph_status sph_cell_sort_noalloc(const sph_params *p, long long n,
                                 const double *x, const double *y,
                                 const double *h, uint64_t *key_out,
                                 uint32_t *perm_out, void *stream);

/* Free all device and host storage of the context: waits for the
 * context's stream, queues the frees on it and waits again, so the memory
 * is back with the device when the call returns (synchronises that stream
 * only). */
sph_status sph_destroy(sph_ctx *ctx);

/* Message of the last error on this context ("" if none); valid until the
 * next call on the context.  NULL ctx: message of the last failed
 * sph_create in this thread. */
const char *sph_last_error(const sph_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
