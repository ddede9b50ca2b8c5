// Host side of the library shared by its C ABI units (sph_api.cu: the
// context, rebuild, passes, PEC step, graphs, reads; adapt_api.cu:
// adaptation and the background construction; batch_api.cu: the batched
// step; tune_api.cu: tuning and the autotuner):
// the context, the static particle sets and the helpers the units share.
#pragma once

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "../../include/sph.h"
#include "adapt.cuh"
#include "background.cuh"
#include "lists.cuh"
#include "load_check.cuh"
#include "pair_passes.cuh"
#include "sph_internal.cuh"
#include "team.cuh"

namespace sph {
namespace api {
// Timed kernel families: 0 pass B, 1 pass A, 2 rebuild, 3 PEC stages,
// 4 adaptation, 5 the neighbour walk of the rebuild (k_list_gather), 6 the
// rebuild's keys, sort and gather.
constexpr int NFAM = 7;

struct Timer {
    std::vector<cudaEvent_t> pool;       // free events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> open[NFAM];
    double ms[NFAM] = {0, 0, 0, 0, 0, 0, 0};
    long long count[NFAM] = {0, 0, 0, 0, 0, 0, 0};
};

// Fields gathered by a rebuild (index into sph_ctx::f / ::falt).  F_DS is
// allocated only in the context that holds the background under
// construction (section 3.3); F_X0..F_P0 only travel within a PEC step.
enum {
    F_X = 0, F_Y, F_U, F_V, F_P, F_RHO, F_M, F_H, F_MMIN, F_MMAX, F_DS,
    F_X0, F_Y0, F_U0, F_V0, F_P0, NF
};
static_assert((int)F_DS == (int)S_DS && (int)F_X0 == (int)NSTATE,
              "state field order shared with the adaptation kernels");

// A particle set that does not move between loads (background, walls),
// kept sorted by its own multi-level cell keys with its own cell table.
struct StaticSet {
    int n = 0, cap = 0;
    double *x = nullptr, *y = nullptr, *h = nullptr;
    double *ex[3] = {nullptr, nullptr, nullptr};   // extra per-particle fields
    int nex = 0;
    float4 *pk = nullptr;       // anchor data (context anchor lattice)
    int pk_version = -1;        // anchor version pk was computed for
    int64_t *id = nullptr;                         // load index
    double *cmin = nullptr;     // background: least ds of each cell, at the
                                // cell's first particle
    uint64_t *key = nullptr, *tkey = nullptr;
    uint32_t *perm = nullptr, *tstart = nullptr, *tend = nullptr;
    float *tmaxh = nullptr;
    int *bbox = nullptr;
    uint32_t *mask = nullptr;
    uint32_t *occ = nullptr;    // occupancy map (OCC_WORDS words)
    uint32_t tmask = 0;
    double c0 = 0.0;
    int lmax = 0, mbits = 1, lbits = 0;
    Level lev[MAX_LEVELS];
    SortScratch sc;
};

}  // namespace api
}  // namespace sph

using sph::api::StaticSet;
using sph::api::Timer;
using sph::api::NFAM;
using namespace sph;
using namespace sph::api;

struct sph_ctx {
    sph_params prm;
    cudaStream_t s = nullptr;
    std::string err;
    long long cap = 0;
    int n = 0;
    Domain dom;
    double c0 = 0.0;
    int lmax = 0, mbits = 1, lbits = 0;
    Level lev[MAX_LEVELS];

    double *f[NF] = {};      // FP64 state, current (sorted) order
    double *falt[NF] = {};   // gather targets, swapped with f
    int64_t *id = nullptr, *id_alt = nullptr;

    // pair-pass outputs and mirrors, sized for doubles (floats use half)
    void *nbA = nullptr, *nbB = nullptr;   // pass-B records (double4 sized)
    void *rhoR = nullptr, *beta = nullptr, *pavg = nullptr, *drx = nullptr,
         *dry = nullptr, *V = nullptr, *rb2 = nullptr, *dpdt = nullptr,
         *dudt = nullptr, *dvdt = nullptr;
    float *mf = nullptr, *pf = nullptr, *uf = nullptr, *vf = nullptr;
    int *nnb = nullptr;

    // neighbour structure
    uint64_t *skey = nullptr;
    uint32_t *perm = nullptr;
    SortScratch sc;
    uint64_t *tkey = nullptr;
    uint32_t *tstart = nullptr, *tend = nullptr;
    float *tmaxh = nullptr;     // per slot: the cell's largest h
    uint32_t tcap = 0, tmask = 0;
    int *bbox = nullptr;
    uint32_t *level_mask = nullptr;
    uint32_t *cnt_tmp = nullptr;   // n + 1 scratch (list totals)
    // neighbour lists and packed per-particle data
    uint8_t *lvl = nullptr;       // level of each particle (sorted order)
    float4 *pk = nullptr;
    uint32_t *own = nullptr, *rev = nullptr, *off = nullptr, *list = nullptr;
    size_t list_cap = 0;
    int *d_overflow = nullptr;
    uint32_t *longq = nullptr, *d_nlong = nullptr;
    uint32_t *stage = nullptr, *lqueue = nullptr, *d_nlq = nullptr;
    uint32_t *lqref = nullptr;      // queued particles' chunk references
    uint32_t stage_w = 64;          // staging row width (entries)
    uint32_t stage_want = 0;        // width to switch to at the next build
    uint32_t *d_max_own = nullptr;  // largest own-entry count of a build
    Anchor an;
    double anchor_A[2] = {0, 0};
    int anchor_version = 0;     // bumped whenever the anchor lattice is set

    // adaptation
    long long next_id = 0;
    uint32_t *tmp_a = nullptr, *tmp_b = nullptr;   // N + 1 each
    int *closest = nullptr;
    float *mh0 = nullptr, *mds = nullptr;   // merge rounds: h at the build, displacement
    float2 *mq = nullptr;                   // merge rounds: FP32 mass bounds
    // fluid particles' wall lists (rebuilt with every neighbour build)
    uint32_t *wcnt = nullptr, *woff = nullptr, *wcur = nullptr, *wlist = nullptr;
    uint32_t *wlongq = nullptr, *d_wnlong = nullptr;
    uint32_t wcap = 0;
    int wall_mode = 0;              // 0: by wall count, 1: cell walk, 2: lists
    bool wall_lists_valid = false;  // the last build made them
    double *d_force = nullptr;   // sph_forces: 8 n_wall + 4 doubles
    int force_cap = 0;           // walls d_force holds
    double *d_mass = nullptr, *d_mass_part = nullptr;  // [2], [256]
    uint32_t *d_aux = nullptr;                         // [4] adapt counters
    uint32_t *h_pin = nullptr;   // 16 pinned host words: adaptation read-backs
    LoadCheckOut *d_load = nullptr;   // checks of a loaded fluid set
    StaticSet bg;     // background particles (section 3.3); extra: ds, m
    // background construction: the background as a particle context of its
    // own (ds carried in F_DS), created on the first sph_background call
    sph_ctx *bgc = nullptr;
    bool bgc_valid = false;   // bgc holds the same set as bg
    bool has_ds = false;      // this context is such a background context
    long long bg_next_id = 0; // id the next background split child receives
    long long adapt_calls = 0;
    double *omega = nullptr;                 // fluid vorticity
    unsigned long long *d_wmax = nullptr;    // max |omega| (bits)
    unsigned long long *d_minmax = nullptr;  // [2] min / max (bits)
    StaticSet wall;   // dummy wall particles (section 2.2); extra: m, u, v
    StaticSet region; // refinement-region markers (section 3.3)
    double *wp = nullptr, *wugx = nullptr, *wugy = nullptr;   // wall BC

    // device scalars
    double *d_dt = nullptr, *d_t = nullptr;
    unsigned long long *d_hmin = nullptr;
    int *d_nonfinite = nullptr;
    uint32_t *d_total = nullptr;

    bool grid_valid = false, rhs_valid = false, have_dt = false;
    // list sizing: entry total and particle count of the last build that
    // read its total back, for exact lists and for lists with a skin
    uint32_t last_total = 0, last_total_skin = 0;
    float skin = 1.0f;          // skin factor of the current lists (1: exact)
    int *d_skin_err = nullptr;  // set when particles outran the skin
    int last_total_n = 0, last_total_skin_n = 0;
    long long steps = 0;
    int launches = 0;
    bool timing = false;
    // launch configuration (sph_set_tuning / sph_autotune)
    double c0_scale = 1.0;
    int walk_choice = 0, team_a = 0, team_b = 0;
    int use_graphs = 1;
    long long cfg_version = 0;   // bumped when the loaded sets or the launch
                                 // configuration change
    int graph_next_drop = 0;
    long long graph_launches = 0;
    long long graph_cfg_seen = -1;   // capture only after two steps with
    int steps_same_cfg = 0;          // no configuration change
    // sph_step's step captured as CUDA graphs, one per buffer assignment the
    // step starts from (a step swaps the state buffers, so two alternate)
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<uintptr_t> key;              // what the launches depend on
        double *f_after[NF], *falt_after[NF];    // buffers after the step
        int64_t *id_after = nullptr, *id_alt_after = nullptr;
        uint32_t tmask = 0;
        float skin = 1.0f;
        int launches = 0;
    } graphs[2];
    Timer tm;
};

namespace sph {
namespace api {

sph_status fail(sph_ctx *c, sph_status st, const std::string &msg);
sph_status cuda_check(sph_ctx *c, const char *where);
void t_begin(sph_ctx *c, int fam, cudaEvent_t *ev);
void t_end(sph_ctx *c, int fam, cudaEvent_t ev0);
void t_collect(sph_ctx *c);
int bits_for(long long v);
Grid make_grid(const sph_ctx *c);
Grid grid_for_kernels(const sph_ctx *c);
ListArgs list_args(sph_ctx *c);
PackArgs pack_args(sph_ctx *c, bool table_end);
void pack(sph_ctx *c, bool table_end);
bool want_wall_lists(const sph_ctx *c);
sph_status rebuild(sph_ctx *c, bool mid_step, bool exact = true,
                          float skin = 1.0f, bool for_walls = true);
WallBcArgs wall_bc_args(sph_ctx *c);
void run_passes(sph_ctx *c);
void run_pec(sph_ctx *c, double f);
void store_rho(sph_ctx *c);
void compute_dt(sph_ctx *c, double *tacc, int nsteps);
void free_ctx(sph_ctx *c);
void ensure_set_pk(sph_ctx *c, StaticSet *S);
bool wall_pk_stale(const sph_ctx *c);
Grid set_grid(const StaticSet &S);
WallView wall_view(const sph_ctx *c);
sph_status setup_fluid_grid(sph_ctx *c, long long n, double hmin,
                                   double hmax);
sph_status check_overflow(sph_ctx *c, const char *who);
std::vector<uintptr_t> graph_key(const sph_ctx *c);
sph_status pec_step(sph_ctx *c, bool exact);
bool graph_step(sph_ctx *c, sph_status *st);
int live_contexts();
void drop_graph(sph_ctx::StepGraph &g);

sph_status compute_vorticity(sph_ctx *c);

// One context's adaptation (sections 3.1-3.4) as phases.  Each phase
// issues its kernels on the context's stream and queues the counts the
// next one needs into the context's pinned words; between phases the
// caller synchronises the stream.  adapt_run drives several contexts in
// lockstep, one synchronisation of all their streams per phase; every
// context gets the kernels, arguments and order of an adaptation of it
// alone.
struct AdaptJob {
    sph_ctx *c = nullptr;
    sph_adapt_stats z;
    cudaEvent_t ev = nullptr;
    sph_status st = SPH_OK;
    enum { SPLIT, MERGE, FINISH, DONE } phase = DONE;
    bool lists_ok = false, first = false, dead = false;
    int n_alive = 0, round = 0;
};
void adapt_run(AdaptJob *jobs, int k);

uint32_t read_u32(sph_ctx *c, const uint32_t *dev, sph_status *st);
uint32_t *pinned_words_get();
void pinned_words_put(uint32_t *p);
sph_status new_ctx(const sph_params *p, cudaStream_t stream, bool has_ds,
                   sph_ctx **out, std::string *why);
sph_status build_set_device(sph_ctx *c, StaticSet *S, long long n,
                                   const double *const *src, int nex,
                                   const int64_t *ids);

// Device buffers of a context come from the stream-ordered allocator on
// the context's stream: allocating and freeing never synchronise the
// device, so creating or destroying one context does not stall the work
// of the others.
template <typename T>
inline bool dalloc(T **p, size_t elems, cudaStream_t s) {
    if (elems == 0) elems = 1;
    return cudaMallocAsync((void **)p, elems * sizeof(T), s) == cudaSuccess;
}
inline void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

inline bool is_mixed(const sph_ctx *c) { return c->prm.precision == SPH_MIXED; }

template <typename R>
inline PassAArgs<R> pass_a_args(sph_ctx *c) {
    PassAArgs<R> a;
    a.n = c->n;
    a.d = c->dom;
    a.an = c->an;
    a.off = c->off;
    a.list = c->list;
    a.pk = c->pk;
    a.x = c->f[F_X];
    a.y = c->f[F_Y];
    a.h = c->f[F_H];
    if (sizeof(R) == sizeof(double)) {
        a.m = (const R *)c->f[F_M];
        a.p = (const R *)c->f[F_P];
        a.u = (const R *)c->f[F_U];
        a.v = (const R *)c->f[F_V];
    } else {
        a.m = (const R *)c->mf;
        a.p = (const R *)c->pf;
        a.u = (const R *)c->uf;
        a.v = (const R *)c->vf;
    }
    a.nbA = (typename V4<R>::T *)c->nbA;
    a.nbB = (typename V4<R>::T *)c->nbB;
    a.rho0 = c->prm.rho0;
    a.w = wall_view(c);
    a.rho = (R *)c->rhoR;
    a.beta = (R *)c->beta;
    a.pavg = (R *)c->pavg;
    a.drx = (R *)c->drx;
    a.dry = (R *)c->dry;
    a.V = (R *)c->V;
    a.rb2 = (R *)c->rb2;
    a.nnb = c->nnb;
    a.filter = c->skin > 1.0f ? 1 : 0;
    return a;
}

template <typename R>
inline PassBArgs<R> pass_b_args(sph_ctx *c, const PassAArgs<R> &a) {
    PassBArgs<R> b;
    b.n = c->n;
    b.d = c->dom;
    b.an = c->an;
    b.off = c->off;
    b.list = c->list;
    b.pk = c->pk;
    b.x = a.x;
    b.y = a.y;
    b.h = a.h;
    b.m = a.m;
    b.p = a.p;
    if (sizeof(R) == sizeof(double)) {
        b.u = (const R *)c->f[F_U];
        b.v = (const R *)c->f[F_V];
    } else {
        b.u = (const R *)c->uf;
        b.v = (const R *)c->vf;
    }
    b.w = a.w;
    b.rho = a.rho;
    b.beta = a.beta;
    b.pavg = a.pavg;
    b.drx = a.drx;
    b.dry = a.dry;
    b.V = a.V;
    b.rb2 = a.rb2;
    b.nbA = a.nbA;
    b.nbB = a.nbB;
    b.dt = c->d_dt;
    b.rho0 = c->prm.rho0;
    b.cs = c->prm.cs;
    b.nu = c->prm.nu;
    b.alpha_e = c->prm.alpha_e;
    b.pavg_mode = c->prm.pavg_mode;
    b.diff_denominator = c->prm.edac_diff_denominator;
    b.rho_factor = c->prm.edac_rho_factor;
    b.dpdt = (R *)c->dpdt;
    b.dudt = (R *)c->dudt;
    b.dvdt = (R *)c->dvdt;
    b.nonfinite = c->d_nonfinite;
    b.filter = a.filter;
    return b;
}

template <typename R>
inline PecArgs<R> pec_args(sph_ctx *c, double f) {
    PecArgs<R> a;
    a.n = c->n;
    a.d = c->dom;
    a.f = f;
    a.save = f < 1.0 ? 1 : 0;   // the predictor starts the step: keep x0..p0
    a.h = c->f[F_H];
    // with skin lists, the predictor's moves must stay within the skin: a
    // pair approaches by at most 2 disp_lim max(h) <= (skin - 1) 3 max(h)
    a.disp_lim = 1.5 * ((double)c->skin - 1.0);
    a.skin_err = (a.save && c->skin > 1.0f) ? c->d_skin_err : nullptr;
    a.dt = c->d_dt;
    a.sponge_w = c->prm.sponge_width > 0 && f >= 1.0 ? c->prm.sponge_width : 0.0;
    a.sponge_x1 = c->dom.lo[0] + c->prm.sponge_width;
    a.sponge_U = c->prm.U_ref;
    a.x0 = c->f[F_X0];
    a.y0 = c->f[F_Y0];
    a.u0 = c->f[F_U0];
    a.v0 = c->f[F_V0];
    a.p0 = c->f[F_P0];
    a.dudt = (const R *)c->dudt;
    a.dvdt = (const R *)c->dvdt;
    a.dpdt = (const R *)c->dpdt;
    a.drx = (const R *)c->drx;
    a.dry = (const R *)c->dry;
    a.x = c->f[F_X];
    a.y = c->f[F_Y];
    a.u = c->f[F_U];
    a.v = c->f[F_V];
    a.p = c->f[F_P];
    return a;
}

}  // namespace api
}  // namespace sph
