// Host orchestration and C ABI (include/sph.h) of the GB300 adaptive WCSPH
// library.  Everything numerical is enqueued on the context's stream as
// the library's own kernels; the host only validates, sizes launches and
// moves buffers.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "adapt.cuh"
#include "background.cuh"
#include "lists.cuh"
#include "pair_passes.cuh"
#include "sph_internal.cuh"
#include "team.cuh"

using namespace sph;

namespace {

// reason of the calling thread's last failed call made without a context
// (sph_create, sph_cell_sort_noalloc): sph_last_error(NULL)
thread_local std::string g_create_error;
static std::atomic<int> g_live_ctx{0};   // contexts made by sph_create, not yet destroyed

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

}  // namespace

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

static void free_set(StaticSet *S) {
    void *ps[] = {S->occ, S->x, S->y, S->h, S->ex[0], S->ex[1], S->ex[2], S->id, S->pk, S->cmin,
                  S->key, S->tkey, S->perm, S->tstart, S->tend, S->tmaxh, S->bbox,
                  S->mask, S->sc.key_alt, S->sc.val_alt, S->sc.counts,
                  S->sc.scan_tmp};
    for (void *p : ps) cudaFree(p);
    *S = StaticSet();
}

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

static Grid set_grid(const StaticSet &S);
static WallView wall_view(const sph_ctx *c);
static void ensure_set_pk(sph_ctx *c, StaticSet *S);

// ------------------------------------------------------------- helpers --
static sph_status fail(sph_ctx *c, sph_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

static sph_status cuda_check(sph_ctx *c, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(c, SPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return SPH_OK;
}

template <typename T>
static bool dalloc(T **p, size_t elems) {
    if (elems == 0) elems = 1;
    return cudaMalloc((void **)p, elems * sizeof(T)) == cudaSuccess;
}

static bool is_mixed(const sph_ctx *c) { return c->prm.precision == SPH_MIXED; }

static void t_begin(sph_ctx *c, int fam, cudaEvent_t *ev) {
    *ev = nullptr;
    if (!c->timing) return;
    if (c->tm.pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->tm.pool.push_back(e);
    }
    *ev = c->tm.pool.back();
    c->tm.pool.pop_back();
    cudaEventRecord(*ev, c->s);
    (void)fam;
}

static void t_end(sph_ctx *c, int fam, cudaEvent_t ev0) {
    if (!c->timing || !ev0) return;
    cudaEvent_t e1;
    if (c->tm.pool.empty()) {
        cudaEventCreate(&e1);
    } else {
        e1 = c->tm.pool.back();
        c->tm.pool.pop_back();
    }
    cudaEventRecord(e1, c->s);
    c->tm.open[fam].push_back({ev0, e1});
}

static void t_collect(sph_ctx *c) {
    for (int f = 0; f < NFAM; ++f) {
        for (auto &pr : c->tm.open[f]) {
            float ms = 0.f;
            cudaEventSynchronize(pr.second);
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            c->tm.ms[f] += ms;
            c->tm.count[f] += 1;
            c->tm.pool.push_back(pr.first);
            c->tm.pool.push_back(pr.second);
        }
        c->tm.open[f].clear();
    }
}

static int bits_for(long long v) {   // bits to represent 0..v
    int b = 0;
    while ((1ll << b) <= v) ++b;
    return b;
}

static Grid make_grid(const sph_ctx *c) {
    Grid g;
    g.occ = nullptr;
    g.tkey = c->tkey;
    g.tstart = c->tstart;
    g.tend = c->tend;
    g.tmask = c->tmask;
    g.tmaxh = c->tmaxh;
    g.level_mask = 0;   // filled by caller from device copy? (see rebuild)
    g.mbits = c->mbits;
    g.nlev = c->lmax + 1;
    g.bbox = c->bbox;
    for (int l = 0; l < MAX_LEVELS; ++l) g.lev[l] = c->lev[l];
    return g;
}

// The occupied-level mask lives on the device; pair kernels read it
// through the Grid by value, so the host fetches it once per rebuild.
// To avoid that synchronisation every level up to lmax is queried; empty
// levels cost one bounding-box test (their box is empty).
static Grid grid_for_kernels(const sph_ctx *c) {
    Grid g = make_grid(c);
    g.level_mask = (c->lmax >= 31) ? 0xffffffffu : ((1u << (c->lmax + 1)) - 1u);
    return g;
}

// ---------------------------------------------------------- the rebuild --
// Keys, stable sort, gather of the state in sorted order, cell table and
// (mixed path) float mirrors.  mid_step: also carry the PEC stage-start
// copies x0..p0.
static ListArgs list_args(sph_ctx *c) {
    ListArgs la;
    la.skin = 1.0f;
    la.n = c->n;
    la.g = grid_for_kernels(c);
    la.d = c->dom;
    la.an = c->an;
    la.x = c->f[F_X];
    la.y = c->f[F_Y];
    la.h = c->f[F_H];
    la.pk = c->pk;
    la.lev = c->lvl;
    la.skey = c->skey;
    la.own = c->own;
    la.rev = c->rev;
    la.off = c->off;
    la.list = c->list;
    la.cap = (uint32_t)std::min<size_t>(c->list_cap, 0xffffffffu);
    la.overflow = c->d_overflow;
    la.longq = c->longq;
    la.nlong = c->d_nlong;
    la.stage = c->stage;
    la.stage_w = c->stage_w;
    la.walk = c->walk_choice;
    la.max_own = c->d_max_own;
    la.queue = c->lqueue;
    la.nqueue = c->d_nlq;
    return la;
}

// Per-particle anchor records (and the mixed path's float mirrors) at the
// current positions; with table_end also the cell ends of the table (part
// of a rebuild).
static PackArgs pack_args(sph_ctx *c, bool table_end) {
    const int n = c->n;
    PackArgs pa;
    pa.n = n;
    pa.lshift = 2 * c->mbits;
    pa.mixed = is_mixed(c) ? 1 : 0;
    pa.skey = c->skey;
    pa.x = c->f[F_X];
    pa.y = c->f[F_Y];
    pa.h = c->f[F_H];
    pa.m = c->f[F_M];
    pa.p = c->f[F_P];
    pa.u = c->f[F_U];
    pa.v = c->f[F_V];
    for (int ax = 0; ax < 2; ++ax) {
        pa.lo[ax] = c->dom.lo[ax];
        pa.Ad[ax] = c->anchor_A[ax];
        pa.invAd[ax] = 1.0 / c->anchor_A[ax];
    }
    pa.an = c->an;
    pa.lev = c->lvl;
    pa.pk = c->pk;
    pa.mf = c->mf;
    pa.pf = c->pf;
    pa.uf = c->uf;
    pa.vf = c->vf;
    pa.tkey = c->tkey;
    pa.tend = table_end ? c->tend : nullptr;
    pa.tmask = c->tmask;
    pa.tmaxh = c->tmaxh;
    return pa;
}
static void pack(sph_ctx *c, bool table_end) {
    launch_pack(c->s, pack_args(c, table_end));
    c->launches += 1;
}

// exact: read the list total back (one synchronisation) and grow the list
// buffer before filling -- unless the last total read back was at most
// half the buffer and the particle count is within 10 % of the one it was
// read at, where the build runs without the synchronisation.  Without it,
// entries past the capacity are dropped and flagged, and the flag is
// checked at the next synchronising call (which then reports
// SPH_ECAPACITY and forces an exact build).
//
// skin > 1: the lists hold every pair with r_ij < skin * 3 max(h_i, h_j), a
// superset of N(i) that stays one while particles move less than
// (skin - 1) 3 max(h) / 2 each.
// Wall lists pay when the walls are many and fine: then the cells of the
// wall grid around a fluid particle are many and mostly empty (measured on
// the cylinders: 12.5k walls at D/1000, passes 7x faster with lists; 578
// walls at D/50, the lists' build costs more than the walks they save).
static bool want_wall_lists(const sph_ctx *c) {
    if (c->wall.n <= 0 || !c->wlist) return false;
    if (c->wall_mode == 1) return false;
    if (c->wall_mode == 2) return true;
    return c->wall.n >= 2048;
}

static sph_status rebuild(sph_ctx *c, bool mid_step, bool exact = true,
                          float skin = 1.0f, bool for_walls = true) {
    const int n = c->n;
    const bool sk = skin > 1.0f;
    const uint32_t lt = sk ? c->last_total_skin : c->last_total;
    const int ltn = sk ? c->last_total_skin_n : c->last_total_n;
    if (exact && lt > 0 && (size_t)lt * 2 <= c->list_cap &&
        (long long)n * 10 <= (long long)ltn * 11 &&
        (long long)n * 10 >= (long long)ltn * 9)
        exact = false;
    if (c->stage_want > c->stage_w) {
        uint32_t *ns = nullptr;
        if (dalloc(&ns, (size_t)c->cap * c->stage_want)) {
            cudaFree(c->stage);   // waits for the last build's use of it
            c->stage = ns;
            c->stage_w = c->stage_want;
        } else {
            cudaGetLastError();   // keep the narrower rows
        }
        c->stage_want = 0;
    }
    cudaEvent_t ev;
    t_begin(c, 2, &ev);
    // table of 2n..4n slots (power of two)
    uint32_t t = 1;
    while (t < 2u * (uint32_t)std::max(n, 1)) t <<= 1;
    c->tmask = t - 1;
    RebuildReset rr;
    rr.bbox = c->bbox;
    rr.level_mask = c->level_mask;
    rr.tkey = c->tkey;
    rr.tslots = t;
    rr.zero[0] = c->d_nlq;
    rr.zero[1] = c->d_max_own;
    rr.zero[2] = c->d_nlong;
    const bool walls = for_walls && want_wall_lists(c);
    rr.zero[3] = walls ? c->wcnt + n : nullptr;
    rr.zero[4] = walls ? c->d_wnlong : nullptr;
    launch_rebuild_reset(c->s, rr, &c->launches);
    cudaEvent_t es;
    t_begin(c, 6, &es);
    launch_keys(c->s, n, c->dom, c->c0, c->lmax, c->mbits, c->lev, c->f[F_X],
                c->f[F_Y], c->f[F_H], c->skey, c->perm, c->level_mask, c->bbox,
                c->rev, walls ? c->wcnt : nullptr, walls ? c->wcur : nullptr);
    c->launches += 1;
    radix_sort(c->s, n, 2 * c->mbits + c->lbits, c->skey, c->perm, c->sc,
               &c->launches);
    GatherList gl;
    memset(&gl, 0, sizeof(gl));
    int last = mid_step ? NF : F_X0;
    for (int k = 0; k < last; ++k) {
        if (!c->f[k]) continue;
        gl.src[gl.nd] = c->f[k];
        gl.dst[gl.nd] = c->falt[k];
        gl.nd++;
    }
    gl.isrc[0] = c->id;
    gl.idst[0] = c->id_alt;
    gl.ni = 1;
    gather_insert(c->s, n, c->perm, gl, c->skey, c->tkey, c->tstart, c->tmask,
                  &c->launches);
    t_end(c, 6, es);
    for (int k = 0; k < last; ++k) std::swap(c->f[k], c->falt[k]);
    std::swap(c->id, c->id_alt);
    pack(c, true);
    ListArgs la = list_args(c);
    la.skin = skin;
    c->skin = skin;
    {
        cudaEvent_t ew;
        t_begin(c, 5, &ew);
        launch_list_walk(c->s, la, &c->launches);
        t_end(c, 5, ew);
    }
    list_offsets(c->s, la, c->sc, c->cnt_tmp, &c->launches);
    // the fluid particles' wall lists, with the same skin
    c->wall_lists_valid = false;
    WallListArgs wa;
    if (walls) {
        ensure_set_pk(c, &c->wall);
        wa.w = wall_view(c);
        wa.g = grid_for_kernels(c);
        wa.d = c->dom;
        wa.an = c->an;
        wa.pk = c->pk;
        wa.reach = std::max(skin, 1.0001f);
        wa.cnt = c->wcnt;
        wa.off = c->woff;
        wa.cur = c->wcur;
        wa.list = c->wlist;
        wa.cap = c->wcap;
        wa.overflow = c->d_overflow;
        wa.longq = c->wlongq;
        wa.nlong = c->d_wnlong;
        launch_wall_lists_count(c->s, n, wa, c->sc, &c->launches);
    }
    bool queue = true;
    if (exact && n > 0) {
        uint32_t total = 0, max_own = 0, wtotal = 0;
        cudaMemcpyAsync(&total, c->off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(&max_own, c->d_max_own, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
        if (walls)
            cudaMemcpyAsync(&wtotal, c->woff + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "rebuild sync");
        if (walls && (size_t)wtotal * 2 > c->wcap) {
            const size_t want = std::min<size_t>(2 * (size_t)wtotal + 4096, 0xffffffffull);
            cudaFree(c->wlist);
            c->wlist = nullptr;
            c->wcap = 0;
            if (!dalloc(&c->wlist, want)) {
                cudaGetLastError();
                return fail(c, SPH_ENOMEM, "wall list allocation failed");
            }
            c->wcap = (uint32_t)want;
            wa.list = c->wlist;
            wa.cap = c->wcap;
            c->cfg_version += 1;
        }
        if (sk) {
            c->last_total_skin = total;
            c->last_total_skin_n = n;
        } else {
            c->last_total = total;
            c->last_total_n = n;
        }
        // widen the staging rows from the next build on, so that particles
        // rarely take the second walk (at most 256 entries a row)
        queue = max_own > c->stage_w;
        if (max_own > c->stage_w && c->stage_w < 256)
            c->stage_want = std::min<uint32_t>(256, (max_own + max_own / 4 + 15) & ~15u);
        // twice the entries found: the next builds skip this read-back
        // (and sph_step can replay its captured graph)
        if ((size_t)total * 2 > c->list_cap) {
            size_t want = 2 * (size_t)total + 1024;
            if (want > 0xffffffffull) want = 0xffffffffull;
            if ((size_t)total > want)
                return fail(c, SPH_ECAPACITY, "neighbour lists exceed 2^32 entries");
            cudaFree(c->list);
            c->list = nullptr;
            if (!dalloc(&c->list, want)) {
                cudaGetLastError();
                c->list_cap = 0;
                return fail(c, SPH_ENOMEM, "neighbour list allocation failed");
            }
            c->list_cap = want;
            la = list_args(c);
            la.skin = skin;
        }
    }
    build_lists_fill(c->s, la, is_mixed(c), queue, &c->launches);
    if (walls) launch_wall_lists_fill(c->s, n, wa, &c->launches);
    c->wall_lists_valid = walls;
    t_end(c, 2, ev);
    c->grid_valid = true;
    c->rhs_valid = false;
    return cuda_check(c, "rebuild");
}

template <typename R>
static PassAArgs<R> pass_a_args(sph_ctx *c) {
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
static PassBArgs<R> pass_b_args(sph_ctx *c, const PassAArgs<R> &a) {
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
static void passes(sph_ctx *c) {
    const PassAArgs<R> a = pass_a_args<R>(c);
    cudaEvent_t ev;
    t_begin(c, 1, &ev);
    launch_pass_a<R>(c->s, a, c->team_a);
    t_end(c, 1, ev);
    const PassBArgs<R> b = pass_b_args<R>(c, a);
    t_begin(c, 0, &ev);
    launch_pass_b<R>(c->s, b, c->team_b);
    t_end(c, 0, ev);
    c->launches += 2;
}

static WallBcArgs wall_bc_args(sph_ctx *c) {
    WallBcArgs wb;
    wb.an = c->an;
    wb.pk = c->pk;
    wb.w = wall_view(c);
    wb.g = grid_for_kernels(c);
    wb.qscale = c->skin;
    wb.d = c->dom;
    wb.x = c->f[F_X];
    wb.y = c->f[F_Y];
    wb.h = c->f[F_H];
    wb.u = c->f[F_U];
    wb.v = c->f[F_V];
    wb.p = c->f[F_P];
    wb.pw = c->wp;
    wb.ugx = c->wugx;
    wb.ugy = c->wugy;
    return wb;
}

static void run_passes(sph_ctx *c) {
    ensure_set_pk(c, &c->wall);
    if (c->wall.n > 0) {
        launch_wall_bc(c->s, wall_bc_args(c));
        c->launches += 1;
    }
    if (is_mixed(c))
        passes<float>(c);
    else
        passes<double>(c);
}

template <typename R>
static PecArgs<R> pec_args(sph_ctx *c, double f) {
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

template <typename R>
static void pec(sph_ctx *c, double f) {
    const PecArgs<R> a = pec_args<R>(c, f);
    cudaEvent_t ev;
    t_begin(c, 3, &ev);
    launch_pec<R>(c->s, a);
    t_end(c, 3, ev);
    c->launches += 1;
}

static void run_pec(sph_ctx *c, double f) {
    if (is_mixed(c))
        pec<float>(c, f);
    else
        pec<double>(c, f);
}

// Latest summation density into the FP64 state (density is recomputed,
// never integrated).
static void store_rho(sph_ctx *c) {
    if (is_mixed(c)) {
        launch_float_to_double(c->s, c->n, (const float *)c->rhoR, c->f[F_RHO]);
        c->launches += 1;
    } else {
        cudaMemcpyAsync(c->f[F_RHO], c->rhoR, sizeof(double) * c->n,
                        cudaMemcpyDeviceToDevice, c->s);
    }
}

static void compute_dt(sph_ctx *c, double *tacc, int nsteps) {
    c->launches += launch_dt(c->s, c->n, c->f[F_H], c->d_hmin, c->prm.U_ref, c->prm.cs,
              c->prm.nu, c->d_dt, tacc, nsteps);
    c->have_dt = true;
}

static void free_ctx(sph_ctx *c) {
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < NF; ++k) {
        cudaFree(c->f[k]);
        cudaFree(c->falt[k]);
    }
    void *ps[] = {c->nbA, c->nbB, c->id, c->id_alt, c->rhoR, c->beta, c->pavg, c->drx,
                  c->dry, c->V, c->rb2, c->dpdt, c->dudt, c->dvdt, c->mf,
                  c->pf, c->uf, c->vf, c->nnb, c->skey, c->perm,
                  c->sc.key_alt, c->sc.val_alt, c->sc.counts, c->sc.scan_tmp,
                  c->tkey, c->tstart, c->tend, c->tmaxh, c->bbox, c->level_mask,
                  c->cnt_tmp, c->d_dt, c->d_t, c->d_hmin, c->d_nonfinite,
                  c->d_total, c->lvl, c->pk, c->own, c->rev, c->off, c->list,
                  c->d_overflow, c->d_skin_err, c->longq, c->d_nlong, c->stage, c->lqueue, c->d_max_own,
                  c->d_nlq, c->tmp_a, c->tmp_b,
                  c->closest, c->mh0, c->mds, c->mq, c->d_mass, c->d_mass_part, c->wp, c->wugx,
                  c->wugy, c->d_aux};
    for (void *p : ps) cudaFree(p);
    cudaFree(c->omega);
    cudaFree(c->d_force);
    cudaFree(c->wcnt);
    cudaFree(c->woff);
    cudaFree(c->wcur);
    cudaFree(c->wlist);
    cudaFree(c->wlongq);
    cudaFree(c->d_wnlong);
    cudaFree(c->d_wmax);
    cudaFree(c->d_minmax);
    if (c->bgc) {
        free_ctx(c->bgc);
        delete c->bgc;
        c->bgc = nullptr;
    }
    free_set(&c->bg);
    free_set(&c->wall);
    free_set(&c->region);
    for (auto e : c->tm.pool) cudaEventDestroy(e);
    for (int f = 0; f < NFAM; ++f)
        for (auto &pr : c->tm.open[f]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
}

// ------------------------------------------------------ static sets --
// Background (section 3.3) and dummy walls (section 2.2): sorted by their
// own cell keys, queried by fluid particles.
//
// build_set_sorted: tmp holds nf = 3 + nex device arrays of n doubles (x,
// y, h, extras) and tid the n ids; both are freed here.  hmin: least h.
static sph_status build_set_sorted(sph_ctx *c, StaticSet *S, long long n,
                                   double hmin, int nex, double *tmp,
                                   int64_t *tid) {
    auto done = [&](sph_status st) {
        cudaStreamSynchronize(c->s);
        cudaFree(tmp);
        cudaFree(tid);
        return st;
    };
    if (n > (1ll << 30)) return done(fail(c, SPH_ECAPACITY, "sph_load_particles: set too large"));
    S->n = 0;
    if (n == 0) return done(SPH_OK);
    double c0 = 3.0 * hmin;
    double Lmax = std::max(c->dom.L[0], c->dom.L[1]);
    int lmax = 0;
    while (ldexp(c0, lmax) < Lmax) ++lmax;
    if (lmax >= MAX_LEVELS) return done(fail(c, SPH_EINVAL, "set spans too many cell levels"));
    Level lev[MAX_LEVELS];
    compute_levels(c->dom, c0, lev);
    long long nmax = std::max(lev[0].n[0], lev[0].n[1]);
    if (nmax >= (1ll << MAX_MORTON_BITS)) return done(fail(c, SPH_EINVAL, "set grid too fine"));
    if (n > S->cap || nex != S->nex) {
        free_set(S);
        size_t N = (size_t)n;
        bool ok = dalloc(&S->x, N) && dalloc(&S->y, N) && dalloc(&S->h, N) &&
                  dalloc(&S->id, N) && dalloc(&S->key, N) && dalloc(&S->perm, N) &&
                  dalloc(&S->pk, N) &&
                  dalloc(&S->bbox, MAX_LEVELS * 4) && dalloc(&S->mask, 1) &&
                  dalloc(&S->occ, OCC_WORDS) &&
                  dalloc(&S->sc.key_alt, N) && dalloc(&S->sc.val_alt, N);
        for (int k = 0; k < nex; ++k) ok = ok && dalloc(&S->ex[k], N);
        ok = ok && dalloc(&S->cmin, N);
        size_t tiles = (N + 2047) / 2048;
        S->sc.counts_cap = 256 * tiles;
        S->sc.scan_cap = scan_scratch_elems(S->sc.counts_cap);
        ok = ok && dalloc(&S->sc.counts, S->sc.counts_cap) &&
             dalloc(&S->sc.scan_tmp, S->sc.scan_cap);
        uint32_t t = 1;
        while (t < 2u * (uint32_t)N) t <<= 1;
        ok = ok && dalloc(&S->tkey, t) && dalloc(&S->tstart, t) && dalloc(&S->tend, t) &&
             dalloc(&S->tmaxh, t);
        if (!ok) {
            cudaGetLastError();
            free_set(S);
            return done(fail(c, SPH_ENOMEM, "particle set allocation failed"));
        }
        S->cap = (int)n;
        S->nex = nex;
    }
    const int nf = 3 + nex;
    S->c0 = c0;
    S->lmax = lmax;
    memcpy(S->lev, lev, sizeof(lev));
    S->mbits = std::max(1, bits_for(nmax - 1));
    S->lbits = bits_for(lmax);
    launch_reset_bbox(c->s, S->bbox, S->mask);
    launch_keys(c->s, (int)n, c->dom, c0, lmax, S->mbits, S->lev, tmp, tmp + n,
                tmp + 2 * n, S->key, S->perm, S->mask, S->bbox);
    launch_occupancy(c->s, (int)n, S->key, 2 * S->mbits, S->bbox, S->occ,
                     &c->launches);
    radix_sort(c->s, (int)n, 2 * S->mbits + S->lbits, S->key, S->perm, S->sc,
               &c->launches);
    GatherList gl;
    memset(&gl, 0, sizeof(gl));
    double *dst[6] = {S->x, S->y, S->h, S->ex[0], S->ex[1], S->ex[2]};
    for (int k = 0; k < nf; ++k) {
        gl.src[k] = tmp + (size_t)k * n;
        gl.dst[k] = dst[k];
    }
    gl.nd = nf;
    gl.isrc[0] = tid;
    gl.idst[0] = S->id;
    gl.ni = 1;
    gather_by_perm(c->s, (int)n, S->perm, gl, &c->launches);
    uint32_t t = 1;
    while (t < 2u * (uint32_t)n) t <<= 1;
    S->tmask = t - 1;
    build_cell_table(c->s, (int)n, S->key, S->tkey, S->tstart, S->tend, S->tmask,
                     &c->launches, S->h, S->tmaxh);
    if (nex > 0) launch_cell_min(c->s, (int)n, S->key, S->ex[0], S->cmin, &c->launches);
    c->launches += 2;
    done(SPH_OK);
    S->n = (int)n;
    S->pk_version = -1;
    return cuda_check(c, "build_set");
}

// From host arrays (validated here); ids NULL: 0..n-1.
static sph_status build_set(sph_ctx *c, StaticSet *S, long long n,
                            const double *x, const double *y, const double *h,
                            const double *const *extra, int nex,
                            const int64_t *ids) {
    double hmin = INFINITY;
    for (long long i = 0; i < n; ++i) {
        if (!(h[i] > 0) || !isfinite(h[i]) || !isfinite(x[i]) || !isfinite(y[i]))
            return fail(c, SPH_EINVAL, "sph_load_particles: h must be positive, positions finite");
        hmin = std::min(hmin, h[i]);
    }
    if (n == 0) {
        S->n = 0;
        return SPH_OK;
    }
    const int nf = 3 + nex;
    double *tmp = nullptr;
    int64_t *tid = nullptr;
    if (!dalloc(&tmp, (size_t)nf * n) || !dalloc(&tid, (size_t)n)) {
        cudaGetLastError();
        cudaFree(tmp);
        return fail(c, SPH_ENOMEM, "particle set staging allocation failed");
    }
    std::vector<int64_t> idv;
    if (!ids) {
        idv.resize((size_t)n);
        for (long long i = 0; i < n; ++i) idv[i] = i;
        ids = idv.data();
    }
    const double *srcs[6] = {x, y, h, nullptr, nullptr, nullptr};
    for (int k = 0; k < nex; ++k) srcs[3 + k] = extra[k];
    for (int k = 0; k < nf; ++k)
        cudaMemcpyAsync(tmp + (size_t)k * n, srcs[k], sizeof(double) * n,
                        cudaMemcpyHostToDevice, c->s);
    cudaMemcpyAsync(tid, ids, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->s);
    return build_set_sorted(c, S, n, hmin, nex, tmp, tid);
}

// From device arrays of another context (x, y, h, extras, ids).
static sph_status build_set_device(sph_ctx *c, StaticSet *S, long long n,
                                   const double *const *src, int nex,
                                   const int64_t *ids) {
    if (n == 0) {
        S->n = 0;
        return SPH_OK;
    }
    const int nf = 3 + nex;
    double *tmp = nullptr;
    int64_t *tid = nullptr;
    if (!dalloc(&tmp, (size_t)nf * n) || !dalloc(&tid, (size_t)n)) {
        cudaGetLastError();
        cudaFree(tmp);
        return fail(c, SPH_ENOMEM, "particle set staging allocation failed");
    }
    for (int k = 0; k < nf; ++k)
        cudaMemcpyAsync(tmp + (size_t)k * n, src[k], sizeof(double) * n,
                        cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(tid, ids, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, c->s);
    launch_minmax_pos(c->s, (int)n, tmp + 2 * n, c->d_minmax);
    c->launches += 1;
    unsigned long long mm[2] = {0, 0};
    cudaMemcpyAsync(mm, c->d_minmax, sizeof(mm), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) {
        cudaFree(tmp);
        cudaFree(tid);
        return cuda_check(c, "build_set_device");
    }
    double hmin;
    memcpy(&hmin, &mm[0], sizeof(double));
    return build_set_sorted(c, S, n, hmin, nex, tmp, tid);
}

// Anchor data of a static set for the context's current anchor lattice.
static void ensure_set_pk(sph_ctx *c, StaticSet *S) {
    if (S->n <= 0 || c->anchor_version == 0 || S->pk_version == c->anchor_version)
        return;
    launch_anchor_pack(c->s, S->n, S->x, S->y, S->h, c->dom.lo, c->anchor_A,
                       c->an, S->pk);
    c->launches += 1;
    S->pk_version = c->anchor_version;
}

static bool wall_pk_stale(const sph_ctx *c) {
    return c->wall.n > 0 && c->anchor_version != 0 && c->wall.pk_version != c->anchor_version;
}

static Grid set_grid(const StaticSet &S) {
    Grid g;
    g.occ = S.occ;
    g.tkey = S.tkey;
    g.tstart = S.tstart;
    g.tend = S.tend;
    g.tmask = S.tmask;
    g.tmaxh = S.tmaxh;
    g.level_mask = (S.lmax >= 31) ? 0xffffffffu : ((1u << (S.lmax + 1)) - 1u);
    g.mbits = S.mbits;
    g.nlev = S.lmax + 1;
    g.bbox = S.bbox;
    for (int l = 0; l < MAX_LEVELS; ++l) g.lev[l] = S.lev[l];
    return g;
}

static WallView wall_view(const sph_ctx *c) {
    WallView w;
    w.n = c->wall.n;
    w.g = set_grid(c->wall);
    w.x = c->wall.x;
    w.y = c->wall.y;
    w.h = c->wall.h;
    w.m = c->wall.ex[0];
    w.uw = c->wall.ex[1];
    w.vw = c->wall.ex[2];
    w.pk = c->wall.pk;
    w.p = c->wp;
    w.ugx = c->wugx;
    w.ugy = c->wugy;
    w.woff = c->wall_lists_valid ? c->woff : nullptr;
    w.wlist = c->wall_lists_valid ? c->wlist : nullptr;
    return w;
}

static sph_status load_background(sph_ctx *c, long long n, const sph_particles *src) {
    if (n > 0 && (!src->x || !src->y || !src->h))
        return fail(c, SPH_EINVAL, "sph_load_particles: background needs x, y, h");
    if (n > 0 && !src->ds && !(c->prm.ds_max > 0))
        return fail(c, SPH_EINVAL, "sph_load_particles: background needs ds (or ds_max > 0)");
    std::vector<double> dsv;
    const double *ds = n > 0 ? src->ds : nullptr;
    if (n > 0 && !ds) {
        dsv.assign((size_t)n, c->prm.ds_max);
        ds = dsv.data();
    }
    for (long long i = 0; i < n; ++i)
        if (!(ds[i] > 0) || !isfinite(ds[i]))
            return fail(c, SPH_EINVAL, "sph_load_particles: background ds must be positive");
    std::vector<double> mv;
    const double *m = n > 0 ? src->m : nullptr;
    if (n > 0 && !m) {
        mv.resize((size_t)n);
        for (long long i = 0; i < n; ++i) mv[i] = c->prm.rho0 * ds[i] * ds[i];
        m = mv.data();
    }
    for (long long i = 0; i < n; ++i)
        if (!(m[i] > 0) || !isfinite(m[i]))
            return fail(c, SPH_EINVAL, "sph_load_particles: background m must be positive");
    const double *ex[2] = {ds, m};
    c->bgc_valid = false;
    c->bg_next_id = n;
    if (n > 0 && src->id) {
        long long mx = -1;
        for (long long i = 0; i < n; ++i) mx = std::max<long long>(mx, src->id[i]);
        c->bg_next_id = mx + 1;
    }
    return build_set(c, &c->bg, n, n ? src->x : nullptr, n ? src->y : nullptr,
                     n ? src->h : nullptr, ex, 2, n ? src->id : nullptr);
}

static sph_status load_walls(sph_ctx *c, long long n, const sph_particles *src) {
    if (n > 0 && (!src->x || !src->y || !src->h || !src->m))
        return fail(c, SPH_EINVAL, "sph_load_particles: walls need x, y, h, m");
    for (long long i = 0; i < n; ++i)
        if (!(src->m[i] > 0) || !isfinite(src->m[i]))
            return fail(c, SPH_EINVAL, "sph_load_particles: wall masses must be positive");
    std::vector<double> zero((size_t)std::max(n, 1ll), 0.0);
    const double *ex[3] = {n ? src->m : nullptr, (n && src->u) ? src->u : zero.data(),
                           (n && src->v) ? src->v : zero.data()};
    sph_status st = build_set(c, &c->wall, n, n ? src->x : nullptr,
                              n ? src->y : nullptr, n ? src->h : nullptr, ex, 3,
                              nullptr);
    if (st != SPH_OK) return st;
    cudaFree(c->wp);
    cudaFree(c->wugx);
    cudaFree(c->wugy);
    c->wp = c->wugx = c->wugy = nullptr;
    cudaFree(c->wlist);
    c->wlist = nullptr;
    c->wcap = 0;
    const size_t wcap = std::max<size_t>(4096, 256 * (size_t)n);
    if (n > 0 && !(dalloc(&c->wp, n) && dalloc(&c->wugx, n) && dalloc(&c->wugy, n) &&
                   dalloc(&c->wlist, wcap))) {
        cudaGetLastError();
        c->wall.n = 0;
        return fail(c, SPH_ENOMEM, "wall allocation failed");
    }
    if (n > 0) c->wcap = (uint32_t)wcap;
    c->grid_valid = false;   // the fluid's wall lists must be rebuilt
    c->rhs_valid = false;
    return SPH_OK;
}

static uint32_t read_u32(sph_ctx *c, const uint32_t *dev, sph_status *st) {
    uint32_t v = 0;
    cudaMemcpyAsync(&v, dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) *st = cuda_check(c, "sync");
    return v;
}

// Allocate a context for p->capacity particles (parameters already
// validated).  has_ds: the context holds a background under construction.
static sph_status new_ctx(const sph_params *p, cudaStream_t stream, bool has_ds,
                          sph_ctx **out, std::string *why) {
    sph_ctx *c = new sph_ctx();
    c->prm = *p;
    c->has_ds = has_ds;
    c->s = stream;
    c->cap = p->capacity;
    for (int a = 0; a < 2; ++a) {
        c->dom.lo[a] = p->lo[a];
        c->dom.hi[a] = p->hi[a];
        c->dom.L[a] = p->hi[a] - p->lo[a];
        c->dom.half[a] = 0.5 * c->dom.L[a];
        c->dom.periodic[a] = p->periodic[a] ? 1 : 0;
    }
    const size_t N = (size_t)c->cap;
    bool ok = true;
    for (int k = 0; k < NF; ++k)
        if (k != F_DS || has_ds) ok = ok && dalloc(&c->f[k], N) && dalloc(&c->falt[k], N);
    ok = ok && dalloc(&c->omega, N) && dalloc(&c->d_wmax, 1) && dalloc(&c->d_minmax, 2);
    ok = ok && dalloc(&c->id, N) && dalloc(&c->id_alt, N);
    double **rs[] = {(double **)&c->rhoR, (double **)&c->beta, (double **)&c->pavg,
                     (double **)&c->drx, (double **)&c->dry, (double **)&c->V,
                     (double **)&c->rb2, (double **)&c->dpdt, (double **)&c->dudt,
                     (double **)&c->dvdt};
    for (auto pp : rs) ok = ok && dalloc(pp, N);
    ok = ok && dalloc((double4_32a **)&c->nbA, N) && dalloc((double4_32a **)&c->nbB, N);
    ok = ok && dalloc(&c->mf, N) && dalloc(&c->pf, N) && dalloc(&c->uf, N) &&
         dalloc(&c->vf, N) && dalloc(&c->nnb, N);
    ok = ok && dalloc(&c->skey, N) && dalloc(&c->perm, N) &&
         dalloc(&c->sc.key_alt, N) && dalloc(&c->sc.val_alt, N);
    size_t tiles = (N + 2047) / 2048;
    c->sc.counts_cap = 256 * tiles;
    c->sc.scan_cap = scan_scratch_elems(std::max(c->sc.counts_cap, N + 1));
    ok = ok && dalloc(&c->sc.counts, c->sc.counts_cap) &&
         dalloc(&c->sc.scan_tmp, c->sc.scan_cap);
    uint32_t t = 1;
    while (t < 2u * (uint32_t)N) t <<= 1;
    c->tcap = t;
    ok = ok && dalloc(&c->tkey, t) && dalloc(&c->tstart, t) && dalloc(&c->tend, t) &&
         dalloc(&c->tmaxh, t);
    ok = ok && dalloc(&c->bbox, MAX_LEVELS * 4) && dalloc(&c->level_mask, 1) &&
         dalloc(&c->cnt_tmp, N + 1);
    ok = ok && dalloc(&c->d_dt, 2) && dalloc(&c->d_t, 1) && dalloc(&c->d_hmin, 1) &&
         dalloc(&c->d_nonfinite, 1) && dalloc(&c->d_total, 1) &&
         dalloc(&c->d_skin_err, 1) &&
         dalloc(&c->d_overflow, 1);
    ok = ok && dalloc(&c->lvl, N) && dalloc(&c->pk, N) && dalloc(&c->own, N) &&
         dalloc(&c->rev, N) && dalloc(&c->off, N + 1) &&
         dalloc(&c->longq, N) && dalloc(&c->d_nlong, 1) &&
         dalloc(&c->stage, N * c->stage_w) && dalloc(&c->lqueue, N) &&
         dalloc(&c->d_nlq, 1) && dalloc(&c->d_max_own, 1);
    ok = ok && dalloc(&c->tmp_a, N + 1) && dalloc(&c->tmp_b, N + 1) &&
         dalloc(&c->closest, N) && dalloc(&c->mh0, N) && dalloc(&c->mds, N) &&
         dalloc(&c->mq, N) &&
         dalloc(&c->wcnt, N + 1) && dalloc(&c->woff, N + 1) && dalloc(&c->wcur, N) &&
         dalloc(&c->wlongq, N) && dalloc(&c->d_wnlong, 1) &&
         dalloc(&c->d_mass, 2) &&
         dalloc(&c->d_mass_part, 256) && dalloc(&c->d_aux, 4);
    c->list_cap = std::min<size_t>(N * 48, 0xffffffffull);
    ok = ok && dalloc(&c->list, c->list_cap);
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        delete c;
        *why = "device allocation failed";
        return SPH_ENOMEM;
    }
    cudaMemsetAsync(c->d_t, 0, sizeof(double), c->s);
    cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->s);
    cudaMemsetAsync(c->d_overflow, 0, sizeof(int), c->s);
    cudaMemsetAsync(c->d_skin_err, 0, sizeof(int), c->s);
    if (cudaGetLastError() != cudaSuccess) {
        free_ctx(c);
        delete c;
        *why = "CUDA error";
        return SPH_ECUDA;
    }
    *out = c;
    return SPH_OK;
}

// Level-0 cell side, cell levels and the FP32 anchor lattice for a fluid
// set whose smoothing lengths span [hmin, hmax] (n may be 0).
static sph_status setup_fluid_grid(sph_ctx *c, long long n, double hmin,
                                   double hmax) {
    // level-0 cell side
    double c0 = c->prm.cell_c0;
    if (!(c0 > 0)) c0 = c->prm.ds_min > 0 ? 3.0 * c->prm.hdx * c->prm.ds_min : 3.0 * hmin;
    c0 *= c->c0_scale;
    if (n == 0 && !(c0 > 0)) c0 = std::max(c->dom.L[0], c->dom.L[1]);
    double Lmax = std::max(c->dom.L[0], c->dom.L[1]);
    int lmax = 0;
    while (ldexp(c0, lmax) < Lmax) ++lmax;
    if (lmax >= MAX_LEVELS)
        return fail(c, SPH_EINVAL, "sph_load_particles: domain spans too many cell levels");
    Level lev[MAX_LEVELS];
    compute_levels(c->dom, c0, lev);
    long long nmax = std::max(lev[0].n[0], lev[0].n[1]);
    if (nmax >= (1ll << MAX_MORTON_BITS))
        return fail(c, SPH_EINVAL, "sph_load_particles: level-0 grid too fine for the domain");
    for (int a = 0; a < 2; ++a)
        if (c->dom.periodic[a] && !(3.0 * hmax < 0.5 * c->dom.L[a]))
            return fail(c, SPH_EINVAL,
                        "sph_load_particles: 3 h_max must be below half a periodic period");
    // anchor lattice of the FP32 separations: side ~ c0, at most 65535 cells
    Anchor an;
    double Ad[2];
    for (int a = 0; a < 2; ++a) {
        double L = c->dom.L[a];
        long long na;
        if (c->dom.periodic[a]) {
            na = std::max(1ll, (long long)floor(L / c0));
            if (na > 65535) na = 65535;
            Ad[a] = L / (double)na;
        } else {
            Ad[a] = std::max(c0, L / 65535.0);
            na = std::max(1ll, (long long)ceil(L / Ad[a]));
            if (na > 65535) na = 65535;
        }
        an.A[a] = (float)Ad[a];
        an.iA[a] = (float)(1.0 / Ad[a]);
        an.n[a] = (int)na;
        an.periodic[a] = c->dom.periodic[a];
    }
    c->an = an;
    c->anchor_A[0] = Ad[0];
    c->anchor_A[1] = Ad[1];
    c->anchor_version += 1;
    c->c0 = c0;
    c->lmax = lmax;
    memcpy(c->lev, lev, sizeof(lev));
    c->mbits = std::max(1, bits_for(nmax - 1));
    c->lbits = bits_for(lmax);
    return SPH_OK;
}

// One split pass (section 3.1): flag m > m_max, scan, rank the parents by
// id, emit the children.  One synchronisation (the parent count).
static sph_status split_pass(sph_ctx *c, uint32_t *count_out) {
    sph_status st = SPH_OK;
    *count_out = 0;
    launch_split_flag(c->s, c->n, c->f[F_M], c->f[F_MMAX], c->tmp_a);
    exclusive_scan(c->s, c->tmp_a, c->tmp_b, c->n, c->d_total, c->sc, &c->launches);
    c->launches += 1;
    uint32_t count = read_u32(c, c->d_total, &st);
    if (st != SPH_OK) return st;
    if ((long long)c->n + 6ll * count > c->cap)
        return fail(c, SPH_ECAPACITY, c->has_ds
                        ? "sph_background: split children exceed bg_capacity"
                        : "sph_adapt: split children exceed the capacity");
    if (count > 0) {
        launch_split_collect(c->s, c->n, c->tmp_a, c->tmp_b, c->id, c->skey, c->perm);
        radix_sort(c->s, (int)count, std::max(1, bits_for(c->next_id)), c->skey,
                   c->perm, c->sc, &c->launches);
        SplitArgs a;
        a.n = c->n;
        a.count = (int)count;
        a.d = c->dom;
        for (int k = 0; k < NSTATE; ++k) a.f[k] = c->f[k];
        a.id = c->id;
        a.parent = c->perm;
        a.next_id = c->next_id;
        a.alpha = c->prm.split_alpha;
        a.eps = c->prm.split_eps;
        launch_split_emit(c->s, a);
        c->launches += 2;
        c->n += 6 * (int)count;
        c->next_id += 6ll * count;
        c->grid_valid = false;
    }
    *count_out = count;
    return SPH_OK;
}

// Arguments of the shift and h-update kernels over the current lists.
static ShiftArgs shift_args(sph_ctx *c) {
    ShiftArgs sa;
    sa.n = c->n;
    sa.d = c->dom;
    for (int k = 0; k < NSTATE; ++k) sa.f[k] = c->f[k];
    sa.off = c->off;
    sa.list = c->list;
    sa.rho0 = c->prm.rho0;
    sa.hdx = c->prm.hdx;
    sa.rho = c->rhoR;
    sa.drx = c->drx;
    sa.dry = c->dry;
    sa.du = c->dudt;
    sa.dv = c->dvdt;
    sa.dp = c->dpdt;
    sa.hnew = c->V;
    sa.w = wall_view(c);
    sa.an = c->an;
    sa.pk = c->pk;
    sa.mf = c->mf;
    sa.uf = c->uf;
    sa.vf = c->vf;
    sa.pf = c->pf;
    sa.filter = 0;
    return sa;
}

// ------------------------------------------------ background construction --
// The background under construction (section 3.3) lives in a context of
// its own (FP64, ds in F_DS), so the fluid's rebuild, split and shift
// machinery serves it unchanged.  It is loaded from the context's
// background set and written back into it after the iterations.
static sph_status ensure_bgc(sph_ctx *c) {
    const long long n = c->bg.n;
    long long cap = c->prm.bg_capacity > 0 ? c->prm.bg_capacity
                                           : std::max(100ll * n, 1ll << 18);
    cap = std::min(std::max(cap, n), 1ll << 30);
    if (c->bgc && c->bgc_valid) return SPH_OK;
    if (c->bgc && c->bgc->cap < cap) {
        free_ctx(c->bgc);
        delete c->bgc;
        c->bgc = nullptr;
    }
    if (!c->bgc) {
        sph_params p = c->prm;
        p.precision = SPH_FP64;
        p.capacity = cap;
        p.cell_c0 = 0.0;
        p.n_bg = 0;
        std::string why;
        sph_status st = new_ctx(&p, c->s, true, &c->bgc, &why);
        if (st != SPH_OK) return fail(c, st, "sph_background: " + why);
    }
    sph_ctx *b = c->bgc;
    launch_minmax_pos(c->s, (int)n, c->bg.h, c->d_minmax);
    c->launches += 1;
    unsigned long long mm[2] = {0, 0};
    cudaMemcpyAsync(mm, c->d_minmax, sizeof(mm), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_background");
    double hmin, hmax;
    memcpy(&hmin, &mm[0], sizeof(double));
    memcpy(&hmax, &mm[1], sizeof(double));
    sph_status st = setup_fluid_grid(b, n, hmin, hmax);
    if (st != SPH_OK) return fail(c, st, b->err);
    b->n = (int)n;
    const size_t bytes = sizeof(double) * n;
    cudaMemcpyAsync(b->f[F_X], c->bg.x, bytes, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(b->f[F_Y], c->bg.y, bytes, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(b->f[F_H], c->bg.h, bytes, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(b->f[F_DS], c->bg.ex[0], bytes, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(b->f[F_M], c->bg.ex[1], bytes, cudaMemcpyDeviceToDevice, c->s);
    cudaMemcpyAsync(b->id, c->bg.id, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, c->s);
    for (int k : {F_U, F_V, F_P, F_RHO, F_MMIN, F_MMAX})
        cudaMemsetAsync(b->f[k], 0, bytes, c->s);
    b->next_id = c->bg_next_id;
    b->grid_valid = b->rhs_valid = b->have_dt = false;
    c->bgc_valid = true;
    return cuda_check(c, "sph_background load");
}

// Fluid vorticity at the current state into c->omega (lists rebuilt).
static sph_status compute_vorticity(sph_ctx *c) {
    sph_status st = rebuild(c, false);
    if (st != SPH_OK) return st;
    VortArgs v;
    v.n = c->n;
    v.d = c->dom;
    v.x = c->f[F_X];
    v.y = c->f[F_Y];
    v.u = c->f[F_U];
    v.v = c->f[F_V];
    v.m = c->f[F_M];
    v.rho = c->f[F_RHO];
    v.h = c->f[F_H];
    v.off = c->off;
    v.list = c->list;
    v.omega = c->omega;
    v.wmax = c->d_wmax;
    launch_vorticity(c->s, v);
    c->launches += 1;
    return SPH_OK;
}

// One construction iteration on the background context b (see
// sph_background in sph.h).  vort: c->omega / c->d_wmax hold the fluid
// vorticity and c's cell structure matches the fluid positions.
static sph_status bg_iteration(sph_ctx *c, sph_ctx *b, bool vort,
                               sph_bg_stats *z) {
    const sph_params &P = c->prm;
    sph_status st;
    if ((st = rebuild(b, false)) != SPH_OK) return fail(c, st, b->err);
    BgMarkArgs ma;
    ma.n = b->n;
    ma.d = b->dom;
    ma.x = b->f[F_X];
    ma.y = b->f[F_Y];
    ma.h = b->f[F_H];
    ma.ds = b->f[F_DS];
    ma.mark = b->tmp_a;
    ma.ds_min = P.ds_min;
    ma.nw = c->wall.n;
    ma.wg = set_grid(c->wall);
    ma.wx = c->wall.x;
    ma.wy = c->wall.y;
    ma.wh = c->wall.h;
    ma.nr = c->region.n;
    ma.rg = set_grid(c->region);
    ma.rx = c->region.x;
    ma.ry = c->region.y;
    ma.rh = c->region.h;
    ma.nf = vort ? c->n : 0;
    ma.fg = grid_for_kernels(c);
    ma.fx = c->f[F_X];
    ma.fy = c->f[F_Y];
    ma.fh = c->f[F_H];
    ma.omega = c->omega;
    ma.wmax = c->d_wmax;
    ma.vort_k = P.vort_k;
    ma.counts = b->d_aux;
    launch_bg_mark(b->s, ma);
    BgSizeArgs sa;
    sa.n = b->n;
    sa.off = b->off;
    sa.list = b->list;
    sa.mark = b->tmp_a;
    sa.ds = b->f[F_DS];
    sa.ds_out = b->falt[F_DS];
    sa.mmin = b->f[F_MMIN];
    sa.mmax = b->f[F_MMAX];
    sa.Cr = P.Cr;
    sa.cr3 = P.Cr * P.Cr * P.Cr;
    sa.ds_min = P.ds_min;
    sa.ds_max = P.ds_max;
    sa.rho0 = P.rho0;
    launch_bg_size(b->s, sa);
    std::swap(b->f[F_DS], b->falt[F_DS]);
    c->launches += 2;
    uint32_t count = 0;
    if ((st = split_pass(b, &count)) != SPH_OK) return fail(c, st, b->err);
    z->n_split += count;
    for (int r = 0; r < P.bg_smooth_iters; ++r) {
        if ((st = rebuild(b, false)) != SPH_OK) return fail(c, st, b->err);
        BgSmoothArgs ha;
        ha.n = b->n;
        ha.off = b->off;
        ha.list = b->list;
        ha.h = b->f[F_H];
        ha.h_out = b->falt[F_H];
        ha.Nr = P.bg_Nr;
        launch_bg_hsmooth(b->s, ha);
        std::swap(b->f[F_H], b->falt[F_H]);
        b->grid_valid = false;
        if ((st = rebuild(b, false)) != SPH_OK) return fail(c, st, b->err);
        launch_shift_round(b->s, shift_args(b), false);
        b->grid_valid = false;
        c->launches += 4;
    }
    return SPH_OK;
}

// Reports (and clears) a neighbour-list overflow of a build that ran
// without its sizing synchronisation, and particles that outran the skin
// of a step's lists; synchronises.
static sph_status check_overflow(sph_ctx *c, const char *who) {
    int flags[2] = {0, 0};
    cudaMemcpyAsync(&flags[0], c->d_overflow, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(&flags[1], c->d_skin_err, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, who);
    if (flags[1]) {
        cudaMemsetAsync(c->d_skin_err, 0, sizeof(int), c->s);
        return fail(c, SPH_ENONFINITE,
                    std::string(who) + ": particles moved farther than the neighbour-list "
                    "skin within one step (flow speed far above U_ref + cs)");
    }
    if (!flags[0]) return SPH_OK;
    cudaMemsetAsync(c->d_overflow, 0, sizeof(int), c->s);
    c->last_total = c->last_total_skin = 0;   // next builds size exactly
    return fail(c, SPH_ECAPACITY, std::string(who) + ": neighbour list overflow");
}

// ================================================================ C ABI ==
template <typename R>
static void forces_launch(sph_ctx *c) {
    ForceArgs<R> a;
    a.w = wall_view(c);
    a.g = grid_for_kernels(c);
    a.d = c->dom;
    a.an = c->an;
    a.pk = c->pk;
    a.x = c->f[F_X];
    a.y = c->f[F_Y];
    a.h = c->f[F_H];
    a.m = c->f[F_M];
    a.u = c->f[F_U];
    a.v = c->f[F_V];
    a.p = c->f[F_P];
    a.rho = (const R *)c->rhoR;
    a.beta = (const R *)c->beta;
    a.rho0 = c->prm.rho0;
    a.nu = c->prm.nu;
    a.fw = c->d_force;
    launch_forces<R>(c->s, a);
}

// One PEC step (section 2.4).  Mixed path: one neighbour build per step,
// with a skin that holds N(i) through the predictor's moves (checked on the
// device; a particle outrunning it is reported at the next
// synchronisation).  FP64 path: a fresh build before each evaluation (wider
// lists would cost more FP64 pair work than the build they save).  exact:
// the first build may read the list size back.
static sph_status pec_step(sph_ctx *c, bool exact) {
    const float step_skin = is_mixed(c) ? 1.1f : 1.0f;
    compute_dt(c, c->d_t, 1);
    sph_status st = rebuild(c, false, exact, step_skin);
    if (st != SPH_OK) return st;
    run_passes(c);
    run_pec(c, 0.5);
    if (step_skin > 1.0f) {
        pack(c, false);   // anchor records and mirrors at the predicted state
    } else {
        st = rebuild(c, true, false);
        if (st != SPH_OK) return st;
    }
    run_passes(c);
    run_pec(c, 1.0);
    store_rho(c);
    c->grid_valid = false;   // positions moved since the last rebuild
    c->rhs_valid = true;     // rates of the n+1/2 evaluation, current order
    c->steps += 1;
    return SPH_OK;
}

// Everything a step's launches depend on besides the device data: the
// buffers (the step swaps them), sizes, list storage, the launch
// configuration and the version of the loaded sets.
static std::vector<uintptr_t> graph_key(const sph_ctx *c) {
    std::vector<uintptr_t> k;
    k.push_back((uintptr_t)c->n);
    for (int f = 0; f < NF; ++f) {
        k.push_back((uintptr_t)c->f[f]);
        k.push_back((uintptr_t)c->falt[f]);
    }
    k.push_back((uintptr_t)c->id);
    k.push_back((uintptr_t)c->id_alt);
    k.push_back((uintptr_t)c->list);
    k.push_back((uintptr_t)c->list_cap);
    k.push_back((uintptr_t)c->stage);
    k.push_back((uintptr_t)c->stage_w);
    k.push_back((uintptr_t)c->cfg_version);
    k.push_back((uintptr_t)c->anchor_version);
    k.push_back((uintptr_t)c->s);
    return k;
}

static void drop_graph(sph_ctx::StepGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
}

// The step as a CUDA graph: captured the first time a buffer assignment
// and configuration comes up, replayed after that (the same kernels with
// the same arguments: results equal the launch-by-launch step bit for
// bit).  Used only when no host decision can arise inside the step: list
// sizes settled (no read-back), staging rows wide enough, timing off, and
// a stream that can be captured.  Returns false (nothing done) when the
// step must run launch by launch; *st reports an error.
static bool graph_step(sph_ctx *c, sph_status *st) {
    *st = SPH_OK;
    const uintptr_t sh = (uintptr_t)c->s;
    if (!c->use_graphs || c->timing || sh <= 2) return false;
    // only while this is the one context of the process: capturing and
    // instantiating a graph wait on other threads' allocations and
    // synchronisations (up to seconds under the serving loop's load)
    if (g_live_ctx.load() > 1) return false;
    // a configuration that changes every step (adaptation between steps)
    // would be captured and thrown away each time: wait for two steps
    if (c->graph_cfg_seen != c->cfg_version) {
        c->graph_cfg_seen = c->cfg_version;
        c->steps_same_cfg = 0;
    }
    if (++c->steps_same_cfg <= 2) return false;
    if (c->stage_want > c->stage_w) return false;
    {   // the build's list size must be known with headroom (no read-back)
        const bool sk = is_mixed(c);
        const uint32_t lt = sk ? c->last_total_skin : c->last_total;
        const int ltn = sk ? c->last_total_skin_n : c->last_total_n;
        const int n = c->n;
        if (!(lt > 0 && (size_t)lt * 2 <= c->list_cap &&
              (long long)n * 10 <= (long long)ltn * 11 &&
              (long long)n * 10 >= (long long)ltn * 9))
            return false;
        if (!is_mixed(c) && !(c->last_total_n > 0)) return false;
    }
    ensure_set_pk(c, &c->wall);
    const std::vector<uintptr_t> key = graph_key(c);
    sph_ctx::StepGraph *g = nullptr;
    for (auto &gg : c->graphs)
        if (gg.exec && gg.key == key) g = &gg;
    if (!g) {
        // a free slot, else the one of another configuration
        sph_ctx::StepGraph *slot = &c->graphs[0];
        for (auto &gg : c->graphs)
            if (!gg.exec) { slot = &gg; break; }
        if (slot->exec) {
            // both slots hold graphs: keep the one the next step will want
            // (the assignment after the step, unknown yet): drop the older
            slot = &c->graphs[c->graph_next_drop];
            c->graph_next_drop ^= 1;
        }
        drop_graph(*slot);
        // capture one step; the host side runs as usual, the kernels only
        // run when the graph is launched below
        double *f0[NF], *fa0[NF];
        memcpy(f0, c->f, sizeof(f0));
        memcpy(fa0, c->falt, sizeof(fa0));
        int64_t *id0 = c->id, *ida0 = c->id_alt;
        const uint32_t tmask0 = c->tmask;
        const float skin0 = c->skin;
        const long long steps0 = c->steps;
        const bool gv0 = c->grid_valid, rv0 = c->rhs_valid;
        const int l0 = c->launches;
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->use_graphs = 0;
            return false;
        }
        sph_status s2 = pec_step(c, false);
        cudaError_t e = cudaStreamEndCapture(c->s, &gr);
        cudaGraphExec_t ex = nullptr;
        if (s2 == SPH_OK && e == cudaSuccess && gr)
            e = cudaGraphInstantiate(&ex, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (s2 != SPH_OK || e != cudaSuccess || !ex) {
            // undo the host side and run the step launch by launch
            cudaGetLastError();
            if (ex) cudaGraphExecDestroy(ex);
            memcpy(c->f, f0, sizeof(f0));
            memcpy(c->falt, fa0, sizeof(fa0));
            c->id = id0;
            c->id_alt = ida0;
            c->tmask = tmask0;
            c->skin = skin0;
            c->steps = steps0;
            c->grid_valid = gv0;
            c->rhs_valid = rv0;
            c->launches = l0;
            c->use_graphs = 0;
            c->err.clear();
            return false;
        }
        slot->exec = ex;
        slot->key = key;
        memcpy(slot->f_after, c->f, sizeof(c->f));
        memcpy(slot->falt_after, c->falt, sizeof(c->falt));
        slot->id_after = c->id;
        slot->id_alt_after = c->id_alt;
        slot->tmask = c->tmask;
        slot->skin = c->skin;
        slot->launches = c->launches - l0;
        g = slot;
    } else {
        memcpy(c->f, g->f_after, sizeof(c->f));
        memcpy(c->falt, g->falt_after, sizeof(c->falt));
        c->id = g->id_after;
        c->id_alt = g->id_alt_after;
        c->tmask = g->tmask;
        c->skin = g->skin;
        c->launches += g->launches;
        c->grid_valid = false;
        c->rhs_valid = true;
        c->steps += 1;
    }
    if (cudaGraphLaunch(g->exec, c->s) != cudaSuccess) *st = cuda_check(c, "sph_step graph");
    c->graph_launches += 1;
    return true;
}

// ============================================================ batches ==
// Several independent simulations advance one PEC step together.  Every
// per-particle phase of the step runs on the batch's stream as one
// persistent launch over the work items of all instances that share a
// precision and a team size (see BatchSpan), and so does the whole
// neighbour build of the small sets whose list sizes are known; the other
// instances build on their own streams.  The bodies are those of the
// single-instance kernels, so with the team sizes an instance uses alone
// its results equal those of sph_step on it alone.
struct sph_batch {
    cudaStream_t s = nullptr;
    int cap = 0;                   // instances per call
    size_t region = 0;             // bytes of one staging region
    char *d_buf = nullptr;         // two device regions (alternating calls)
    char *h_buf = nullptr;         // their pinned host staging
    cudaEvent_t done[2] = {nullptr, nullptr};   // end of a region's last call
    bool used[2] = {false, false};
    cudaEvent_t ev = nullptr;      // fork / join between streams
    int calls = 0;
    int pack_blocks = 0;           // persistent grid of the packing launch
    long long launches = 0;
    // The whole batched step as one CUDA graph, captured once a batch of
    // the same contexts and configurations has come up three times in a
    // row, and replayed while it recurs.  The step swaps each context's
    // state buffers, so two assignments alternate: two slots, each with
    // staging regions of its own (its captured copies read them).
    bool use_graphs = true;
    std::vector<uintptr_t> comp;   // contexts and configurations of the last call
    int same_comp = 0;
    struct Inst {
        double *f_after[NF], *falt_after[NF];
        int64_t *id_after = nullptr, *id_alt_after = nullptr;
        uint32_t tmask = 0;
        float skin = 1.0f;
        int launches = 0;
    };
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<uintptr_t> key;
        std::vector<Inst> inst;
        long long launches = 0;
        char *d = nullptr, *h = nullptr;
    } graphs[2];
    int graph_next_drop = 0;
    long long graph_steps = 0;
};

namespace {

// Argument blocks and work-item offsets, written to pinned memory and
// copied to the same offsets of the device region in stream order.
struct Stager {
    char *h = nullptr, *d = nullptr;
    size_t cap = 0, used = 0, sent = 0;
    template <class T>
    size_t put(const T *p, size_t cnt) {
        used = (used + 15) & ~(size_t)15;
        const size_t o = used, b = sizeof(T) * cnt;
        if (o + b > cap) return (size_t)-1;
        memcpy(h + o, p, b);
        used = o + b;
        return o;
    }
    void flush(cudaStream_t s) {
        if (used > sent)
            cudaMemcpyAsync(d + sent, h + sent, used - sent, cudaMemcpyHostToDevice, s);
        sent = used;
    }
};

// Instances of one phase that share a team size (the key), their argument
// blocks and work-item offsets in the staging region.
struct PhaseGroup {
    int team = 1;
    std::vector<sph_ctx *> cs;
    size_t off_args = 0, off_first = 0;
    int total = 0;
};

// Groups by team (team(c) < 0 or count(c) <= 0: the instance takes no
// part) and stages each group's argument blocks make(c) and offsets.
template <class A, class Team, class Count, class Make>
static bool stage_phase(Stager &st, const std::vector<sph_ctx *> &cs, Team team,
                        Count count, Make make, std::vector<PhaseGroup> &out) {
    out.clear();
    for (sph_ctx *c : cs) {
        const int t = team(c);
        if (t < 0 || count(c) <= 0) continue;
        PhaseGroup *g = nullptr;
        for (auto &x : out)
            if (x.team == t) g = &x;
        if (!g) {
            out.emplace_back();
            g = &out.back();
            g->team = t;
        }
        g->cs.push_back(c);
    }
    for (auto &g : out) {
        std::vector<A> args;
        std::vector<int> first(1, 0);
        const int rows = batch_rows(g.team);
        for (sph_ctx *c : g.cs) {
            args.push_back(make(c));
            first.push_back(first.back() + (count(c) + rows - 1) / rows);
        }
        g.total = first.back();
        g.off_args = st.put(args.data(), args.size());
        g.off_first = st.put(first.data(), first.size());
        if (g.off_args == (size_t)-1 || g.off_first == (size_t)-1) return false;
    }
    return true;
}

static BatchSpan span_of(const Stager &st, const PhaseGroup &g) {
    BatchSpan sp;
    sp.first = (const int *)(st.d + g.off_first);
    sp.k = (int)g.cs.size();
    sp.total = g.total;
    return sp;
}

// One evaluation's staged phases: wall conditions, pass A, pass B and the
// PEC stage that follows, for both precisions.
struct EvalStage {
    std::vector<PhaseGroup> wall, a32, a64, b32, b64, pec32, pec64;
};

// Team size of a batch's pass A / pass B: the one sph_set_tuning set on the
// context, else the size rule applied to the particles of all the batch's
// instances of that precision (they share the GPU: a warp per particle
// that fills it for one small set would idle most lanes in a large batch).
static int batch_team(const std::vector<sph_ctx *> &cs) {
    long long n = 0;
    for (sph_ctx *c : cs) n += c->n;
    return team_size((int)std::min<long long>(n, 1 << 30));
}

template <typename R>
static bool stage_passes(Stager &st, const std::vector<sph_ctx *> &cs,
                         std::vector<PhaseGroup> &ga, std::vector<PhaseGroup> &gb) {
    auto na = [](sph_ctx *c) { return c->n; };
    const int bt = batch_team(cs);
    auto pick = [bt](int t) { return (t == 1 || t == 4 || t == 16 || t == 32) ? t : bt; };
    bool ok = stage_phase<PassAArgs<R>>(
        st, cs, [&](sph_ctx *c) { return pick(c->team_a); }, na,
        [](sph_ctx *c) { return pass_a_args<R>(c); }, ga);
    ok = ok && stage_phase<PassBArgs<R>>(
        st, cs, [&](sph_ctx *c) { return pick(c->team_b); }, na,
        [](sph_ctx *c) { return pass_b_args<R>(c, pass_a_args<R>(c)); }, gb);
    return ok;
}

template <typename R>
static bool stage_pec(Stager &st, const std::vector<sph_ctx *> &cs, double f,
                      std::vector<PhaseGroup> &g) {
    return stage_phase<PecArgs<R>>(
        st, cs, [](sph_ctx *) { return 1; }, [](sph_ctx *c) { return c->n; },
        [f](sph_ctx *c) { return pec_args<R>(c, f); }, g);
}

static bool stage_eval(Stager &st, const std::vector<sph_ctx *> &m32,
                       const std::vector<sph_ctx *> &m64,
                       const std::vector<sph_ctx *> &all, double f, EvalStage &e) {
    bool ok = stage_phase<WallBcArgs>(
        st, all, [](sph_ctx *c) { return c->wall.n > 0 ? team_size(c->wall.n) : -1; },
        [](sph_ctx *c) { return c->wall.n; }, [](sph_ctx *c) { return wall_bc_args(c); },
        e.wall);
    ok = ok && stage_passes<float>(st, m32, e.a32, e.b32);
    ok = ok && stage_passes<double>(st, m64, e.a64, e.b64);
    ok = ok && stage_pec<float>(st, m32, f, e.pec32);
    ok = ok && stage_pec<double>(st, m64, f, e.pec64);
    return ok;
}

static void launch_eval(sph_batch *b, const Stager &st, const EvalStage &e) {
    for (auto &g : e.wall)
        launch_wall_bc_batch(b->s, g.team, (const WallBcArgs *)(st.d + g.off_args), span_of(st, g));
    for (auto &g : e.a32)
        launch_pass_a_batch<float>(b->s, g.team, (const PassAArgs<float> *)(st.d + g.off_args),
                                   span_of(st, g));
    for (auto &g : e.a64)
        launch_pass_a_batch<double>(b->s, g.team, (const PassAArgs<double> *)(st.d + g.off_args),
                                    span_of(st, g));
    for (auto &g : e.b32)
        launch_pass_b_batch<float>(b->s, g.team, (const PassBArgs<float> *)(st.d + g.off_args),
                                   span_of(st, g));
    for (auto &g : e.b64)
        launch_pass_b_batch<double>(b->s, g.team, (const PassBArgs<double> *)(st.d + g.off_args),
                                    span_of(st, g));
    for (auto &g : e.pec32)
        launch_pec_batch<float>(b->s, (const PecArgs<float> *)(st.d + g.off_args), span_of(st, g));
    for (auto &g : e.pec64)
        launch_pec_batch<double>(b->s, (const PecArgs<double> *)(st.d + g.off_args), span_of(st, g));
    b->launches += (long long)(e.wall.size() + e.a32.size() + e.a64.size() + e.b32.size() +
                               e.b64.size() + e.pec32.size() + e.pec64.size());
}

// the contexts' streams wait for the batch stream's work so far
static void fork_to(sph_batch *b, const std::vector<sph_ctx *> &cs) {
    cudaEventRecord(b->ev, b->s);
    for (sph_ctx *c : cs)
        if (c->s != b->s) cudaStreamWaitEvent(c->s, b->ev, 0);
}
// the batch stream waits for the contexts' streams' work so far
static void join_from(sph_batch *b, const std::vector<sph_ctx *> &cs) {
    for (sph_ctx *c : cs) {
        if (c->s == b->s) continue;
        cudaEventRecord(b->ev, c->s);
        cudaStreamWaitEvent(b->s, b->ev, 0);
    }
}

// Staging bytes one instance can need in a call (two evaluations).
static size_t batch_bytes_per_instance() {
    const size_t r = 16;
    auto up = [r](size_t v) { return (v + r - 1) / r * r; };
    const size_t eval = up(sizeof(WallBcArgs)) + up(sizeof(PassAArgs<double>)) +
                        up(sizeof(PassBArgs<double>)) + up(sizeof(PecArgs<double>));
    // a batched small-set build (two for FP64 contexts: one mid-step)
    const size_t build = up(sizeof(DtSmallRec)) + up(sizeof(RebuildReset)) +
                         up(sizeof(KeysRec)) + up(sizeof(RadixSmallRec)) +
                         up(sizeof(GatherInsertRec)) + up(sizeof(PackArgs)) +
                         3 * up(sizeof(ListArgs)) + up(sizeof(ScanSmallRec)) +
                         2 * up(sizeof(SortSegRec));
    return 2 * eval + 2 * build + up(sizeof(PackArgs)) + up(sizeof(RhoStoreArgs));
}

}  // namespace


// ------------------------------------------ batched builds of small sets --
// A context whose build can run in the batched small-set build: the
// single-block sort, scan and time-step kernels take it, its walk is the
// team walk, it has no wall lists, library timing is off, and its list
// sizes are known (the build needs no read-back).  Then the build is the
// one rebuild() makes without read-back, kernel for kernel.
static bool small_build_ok(sph_ctx *c, float skin) {
    const int n = c->n;
    if (n < 2 || n > radix_small_max() || n > scan_small_max() || n > dt_small_max()) return false;
    if (!radix_small_available() || want_wall_lists(c) || c->timing) return false;
    if (c->stage_want > c->stage_w) return false;
    if (2 * c->mbits + c->lbits <= 0) return false;
    const bool sk = skin > 1.0f;
    const uint32_t lt = sk ? c->last_total_skin : c->last_total;
    const int ltn = sk ? c->last_total_skin_n : c->last_total_n;
    if (!(lt > 0 && (size_t)lt * 2 <= c->list_cap && (long long)n * 10 <= (long long)ltn * 11 &&
          (long long)n * 10 >= (long long)ltn * 9))
        return false;
    ListArgs la = list_args(c);
    la.skin = skin;
    return list_walk_kind(la) == 1;
}

// The records of one context's small-set build (and, with_dt, its time
// step), with the host side of rebuild() done: table size, buffer swaps,
// skin and validity flags.
struct SmallBuild {
    sph_ctx *c;
    DtSmallRec dt;
    RebuildReset rr;
    KeysRec keys;
    RadixSmallRec rs;
    GatherInsertRec gi;
    PackArgs pack;
    ListArgs la;
    ScanSmallRec scan;
    SortSegRec seg;
};

static void plan_small_build(sph_ctx *c, bool mid_step, float skin, bool with_dt,
                             SmallBuild &B) {
    const int n = c->n;
    B.c = c;
    if (with_dt) {
        B.dt.n = n;
        B.dt.h = c->f[F_H];
        B.dt.U = c->prm.U_ref;
        B.dt.cs = c->prm.cs;
        B.dt.nu = c->prm.nu;
        B.dt.hmin_bits = c->d_hmin;
        B.dt.dt = c->d_dt;
        B.dt.tacc = c->d_t;
        B.dt.nsteps = 1;
        c->have_dt = true;
    }
    uint32_t t = 1;
    while (t < 2u * (uint32_t)n) t <<= 1;
    c->tmask = t - 1;
    B.rr.bbox = c->bbox;
    B.rr.level_mask = c->level_mask;
    B.rr.tkey = c->tkey;
    B.rr.tslots = t;
    B.rr.zero[0] = c->d_nlq;
    B.rr.zero[1] = c->d_max_own;
    B.rr.zero[2] = c->d_nlong;
    B.rr.zero[3] = nullptr;
    B.rr.zero[4] = nullptr;
    B.keys = make_keys_rec(n, c->dom, c->c0, c->lmax, c->mbits, c->lev, c->f[F_X], c->f[F_Y],
                           c->f[F_H], c->skey, c->perm, c->level_mask, c->bbox, c->rev, nullptr,
                           nullptr);
    B.rs.n = n;
    B.rs.passes = (2 * c->mbits + c->lbits + 7) / 8;
    B.rs.ka = c->skey;
    B.rs.va = c->perm;
    B.rs.kb = c->sc.key_alt;
    B.rs.vb = c->sc.val_alt;
    GatherList &gl = B.gi.g;
    memset(&gl, 0, sizeof(gl));
    const int last = mid_step ? NF : F_X0;
    for (int k = 0; k < last; ++k) {
        if (!c->f[k]) continue;
        gl.src[gl.nd] = c->f[k];
        gl.dst[gl.nd] = c->falt[k];
        gl.nd++;
    }
    gl.isrc[0] = c->id;
    gl.idst[0] = c->id_alt;
    gl.ni = 1;
    B.gi.n = n;
    B.gi.perm = c->perm;
    B.gi.skey = c->skey;
    B.gi.tkey = c->tkey;
    B.gi.tstart = c->tstart;
    B.gi.tmask = c->tmask;
    for (int k = 0; k < last; ++k) std::swap(c->f[k], c->falt[k]);
    std::swap(c->id, c->id_alt);
    B.pack = pack_args(c, true);
    B.la = list_args(c);
    B.la.skin = skin;
    c->skin = skin;
    B.scan.in = c->own;
    B.scan.rev = c->rev;
    B.scan.out = c->off;
    B.scan.n = n;
    B.scan.total_dev = nullptr;
    B.scan.write_total_at_n = 1;
    B.seg.n = n;
    B.seg.off = c->off;
    B.seg.own = c->own;
    B.seg.list = c->list;
    B.seg.cap = B.la.cap;
    B.seg.longq = c->longq;
    B.seg.nlong = c->d_nlong;
    c->wall_lists_valid = false;
    c->grid_valid = true;
    c->rhs_valid = false;
    // (its launches are the batch's: sph_batch_launches counts them)
}

namespace {
// One group of a staged phase with explicit work items an instance.
template <class A>
static bool stage_group(Stager &st, const std::vector<A> &recs, const std::vector<int> &items,
                        int team, PhaseGroup &g) {
    g.team = team;
    g.cs.assign(recs.size(), nullptr);
    std::vector<int> first(1, 0);
    for (int v : items) first.push_back(first.back() + v);
    g.total = first.back();
    g.off_args = st.put(recs.data(), recs.size());
    g.off_first = st.put(first.data(), first.size());
    return g.off_args != (size_t)-1 && g.off_first != (size_t)-1;
}
static int nblk_h(int n, int bs) { return (n + bs - 1) / bs; }
}  // namespace

// The batched build of the contexts in bs (each planned by
// plan_small_build), as one launch per kernel of the build (per team size
// for the team kernels) on the batch stream.
static bool launch_small_builds(sph_batch *b, Stager &st, const std::vector<SmallBuild> &bs,
                                bool with_dt) {
    if (bs.empty()) return true;
    std::vector<DtSmallRec> dt;
    std::vector<RebuildReset> rr;
    std::vector<KeysRec> keys;
    std::vector<RadixSmallRec> rs;
    std::vector<GatherInsertRec> gi;
    std::vector<PackArgs> pk;
    std::vector<ScanSmallRec> sc;
    std::vector<SortSegRec> seg;
    std::vector<int> i_one, i_rr, i_256, i_128, i_fq, i_sl;
    int max_n = 0;
    for (const SmallBuild &B : bs) {
        const int n = B.c->n;
        max_n = std::max(max_n, n);
        if (with_dt) dt.push_back(B.dt);
        rr.push_back(B.rr);
        keys.push_back(B.keys);
        rs.push_back(B.rs);
        gi.push_back(B.gi);
        pk.push_back(B.pack);
        sc.push_back(B.scan);
        seg.push_back(B.seg);
        i_one.push_back(1);
        i_rr.push_back(rebuild_reset_blocks(B.rr.tslots));
        i_256.push_back(nblk_h(n, 256));
        i_128.push_back(nblk_h(n, BATCH_THREADS));
        i_fq.push_back(fill_queue_blocks());
        i_sl.push_back(sort_long_blocks(n));
    }
    // team walk and placement: one group per team size.  The walk's entry
    // order does not depend on its team size, which follows the batch's
    // total like the passes' (see batch_team)
    std::vector<sph_ctx *> bcs;
    for (const SmallBuild &B : bs) bcs.push_back(B.c);
    const int walk_team = batch_team(bcs);
    auto wteam = [walk_team](int) { return walk_team; };
    std::vector<int> walk_teams, place_teams;
    for (const SmallBuild &B : bs) {
        const int tw = wteam(B.c->n), tp = list_place_team(B.c->n);
        if (std::find(walk_teams.begin(), walk_teams.end(), tw) == walk_teams.end())
            walk_teams.push_back(tw);
        if (std::find(place_teams.begin(), place_teams.end(), tp) == place_teams.end())
            place_teams.push_back(tp);
    }
    auto team_group = [&](int team, bool place, PhaseGroup &g) {
        std::vector<ListArgs> la;
        std::vector<int> items;
        for (const SmallBuild &B : bs) {
            const int n = B.c->n;
            const int t = place ? list_place_team(n) : wteam(n);
            if (t != team) continue;
            la.push_back(B.la);
            items.push_back(nblk_h(n * t, 128));
        }
        return stage_group(st, la, items, team, g);
    };
    PhaseGroup gdt, grr, gkeys, grs, ggi, gpk, gsc, gfq, gsr, gsl;
    std::vector<PhaseGroup> gwalk(walk_teams.size()), gplace(place_teams.size());
    bool ok = true;
    if (with_dt) ok = ok && stage_group(st, dt, i_one, 1, gdt);
    ok = ok && stage_group(st, rr, i_rr, 1, grr) && stage_group(st, keys, i_256, 1, gkeys) &&
         stage_group(st, rs, i_one, 1, grs) && stage_group(st, gi, i_256, 1, ggi) &&
         stage_group(st, pk, i_128, 1, gpk) && stage_group(st, sc, i_one, 1, gsc);
    std::vector<ListArgs> la_all;
    for (const SmallBuild &B : bs) la_all.push_back(B.la);
    ok = ok && stage_group(st, la_all, i_fq, 16, gfq) && stage_group(st, seg, i_256, 1, gsr) &&
         stage_group(st, seg, i_sl, 1, gsl);
    for (size_t u = 0; u < walk_teams.size(); ++u) ok = ok && team_group(walk_teams[u], false, gwalk[u]);
    for (size_t u = 0; u < place_teams.size(); ++u) ok = ok && team_group(place_teams[u], true, gplace[u]);
    if (!ok) return false;
    st.flush(b->s);
    auto sp = [&](const PhaseGroup &g) {
        BatchSpan x;
        x.first = (const int *)(st.d + g.off_first);
        x.k = (int)bs.size();
        x.total = g.total;
        return x;
    };
    auto spk = [&](const PhaseGroup &g, int k) {
        BatchSpan x = sp(g);
        x.k = k;
        return x;
    };
    long long nl = 0;
    if (with_dt) {
        launch_dt_small_batch(b->s, (const DtSmallRec *)(st.d + gdt.off_args), sp(gdt));
        ++nl;
    }
    launch_rebuild_reset_batch(b->s, (const RebuildReset *)(st.d + grr.off_args), sp(grr));
    launch_keys_batch(b->s, (const KeysRec *)(st.d + gkeys.off_args), sp(gkeys));
    if (!launch_radix_small_batch(b->s, (const RadixSmallRec *)(st.d + grs.off_args), sp(grs),
                                  max_n))
        return false;
    launch_gather_insert_batch(b->s, (const GatherInsertRec *)(st.d + ggi.off_args), sp(ggi));
    launch_pack_batch(b->s, (const PackArgs *)(st.d + gpk.off_args), sp(gpk), b->pack_blocks);
    nl += 5;
    for (size_t u = 0; u < walk_teams.size(); ++u) {
        int k = 0;
        for (const SmallBuild &B : bs) k += wteam(B.c->n) == walk_teams[u];
        launch_list_gather_batch(b->s, walk_teams[u], (const ListArgs *)(st.d + gwalk[u].off_args),
                                 spk(gwalk[u], k));
        ++nl;
    }
    launch_scan_small_batch(b->s, (const ScanSmallRec *)(st.d + gsc.off_args), sp(gsc));
    ++nl;
    for (size_t u = 0; u < place_teams.size(); ++u) {
        int k = 0;
        for (const SmallBuild &B : bs) k += list_place_team(B.c->n) == place_teams[u];
        launch_list_place_batch(b->s, place_teams[u], (const ListArgs *)(st.d + gplace[u].off_args),
                                spk(gplace[u], k));
        ++nl;
    }
    launch_list_fill_queue_batch(b->s, (const ListArgs *)(st.d + gfq.off_args), sp(gfq));
    launch_list_sort_rev_batch(b->s, (const SortSegRec *)(st.d + gsr.off_args), sp(gsr));
    launch_list_sort_long_batch(b->s, (const SortSegRec *)(st.d + gsl.off_args), sp(gsl));
    nl += 3;
    b->launches += nl;
    return true;
}

// One batched step (the work of sph_batch_step between its checks and its
// final fork): per-instance time step and build, then the staged phases.
// *bad names the context an error belongs to.
static sph_status batch_body(sph_batch *b, const std::vector<sph_ctx *> &all,
                             const std::vector<sph_ctx *> &m32,
                             const std::vector<sph_ctx *> &m64, Stager &st,
                             sph_ctx **bad, bool capturing) {
    // 1. time step and the step's neighbour build (as sph_step): small sets
    // whose sizes are known in the batched build on the batch stream, the
    // others on their own streams
    std::vector<sph_ctx *> rest;
    std::vector<SmallBuild> sb;
    for (sph_ctx *c : all) {
        const float skin = is_mixed(c) ? 1.1f : 1.0f;
        if (small_build_ok(c, skin)) {
            sb.emplace_back();
            plan_small_build(c, false, skin, true, sb.back());
        } else {
            rest.push_back(c);
        }
    }
    // work queued on the small sets' streams comes first (a replayed graph
    // is joined by its caller, and inside a capture only captured work
    // may be waited on)
    if (!capturing) {
        std::vector<sph_ctx *> small;
        for (const SmallBuild &B : sb) small.push_back(B.c);
        join_from(b, small);
    }
    fork_to(b, rest);
    for (sph_ctx *c : rest) {
        compute_dt(c, c->d_t, 1);
        sph_status s2 = rebuild(c, false, true, is_mixed(c) ? 1.1f : 1.0f);
        if (s2 != SPH_OK) {
            *bad = c;
            join_from(b, rest);
            return s2;
        }
    }
    if (!launch_small_builds(b, st, sb, true)) {
        join_from(b, rest);
        return fail(all[0], SPH_ECUDA, "sph_batch_step: batched build could not be staged");
    }
    // wall anchor records on the contexts' streams where stale
    for (const SmallBuild &B : sb)
        if (wall_pk_stale(B.c)) rest.push_back(B.c);
    for (sph_ctx *c : all) ensure_set_pk(c, &c->wall);
    join_from(b, rest);
    // 2. predictor evaluation and stage
    *bad = all[0];
    EvalStage e1, e2;
    if (!stage_eval(st, m32, m64, all, 0.5, e1))
        return fail(all[0], SPH_ECUDA, "sph_batch_step: staging overflow");
    std::vector<PhaseGroup> gpack, grho;
    bool ok = stage_phase<PackArgs>(
        st, m32, [](sph_ctx *) { return 1; }, [](sph_ctx *c) { return c->n; },
        [](sph_ctx *c) { return pack_args(c, false); }, gpack);
    ok = ok && stage_phase<RhoStoreArgs>(
        st, m32, [](sph_ctx *) { return 1; }, [](sph_ctx *c) { return c->n; },
        [](sph_ctx *c) {
            RhoStoreArgs a;
            a.n = c->n;
            a.src = (const float *)c->rhoR;
            a.dst = c->f[F_RHO];
            return a;
        }, grho);
    if (!ok) return fail(all[0], SPH_ECUDA, "sph_batch_step: staging overflow");
    const bool fp64 = !m64.empty();
    if (!fp64 && !stage_eval(st, m32, m64, all, 1.0, e2))
        return fail(all[0], SPH_ECUDA, "sph_batch_step: staging overflow");
    st.flush(b->s);
    launch_eval(b, st, e1);
    // 3. mid-step: mixed instances repack at the predicted state (their
    // lists carry a skin); FP64 instances rebuild
    for (auto &g : gpack) {
        launch_pack_batch(b->s, (const PackArgs *)(st.d + g.off_args), span_of(st, g),
                          b->pack_blocks);
        b->launches += 1;
    }
    if (fp64) {
        std::vector<sph_ctx *> rest64;
        std::vector<SmallBuild> sb64;
        for (sph_ctx *c : m64) {
            if (small_build_ok(c, 1.0f)) {
                sb64.emplace_back();
                plan_small_build(c, true, 1.0f, false, sb64.back());
            } else {
                rest64.push_back(c);
            }
        }
        fork_to(b, rest64);
        for (sph_ctx *c : rest64) {
            sph_status s2 = rebuild(c, true, false);
            if (s2 != SPH_OK) {
                *bad = c;
                join_from(b, rest64);
                return s2;
            }
        }
        if (!launch_small_builds(b, st, sb64, false)) {
            join_from(b, rest64);
            return fail(all[0], SPH_ECUDA, "sph_batch_step: batched build could not be staged");
        }
        for (const SmallBuild &B : sb64)
            if (wall_pk_stale(B.c)) rest64.push_back(B.c);
        for (sph_ctx *c : m64) ensure_set_pk(c, &c->wall);
        join_from(b, rest64);
        if (!stage_eval(st, m32, m64, all, 1.0, e2))
            return fail(all[0], SPH_ECUDA, "sph_batch_step: staging overflow");
        st.flush(b->s);
    }
    // 4. corrector evaluation and stage, density into the FP64 state
    launch_eval(b, st, e2);
    for (auto &g : grho) {
        launch_rho_store_batch(b->s, (const RhoStoreArgs *)(st.d + g.off_args), span_of(st, g));
        b->launches += 1;
    }
    for (sph_ctx *c : m64)
        cudaMemcpyAsync(c->f[F_RHO], c->rhoR, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                        b->s);
    for (sph_ctx *c : all) {
        c->grid_valid = false;
        c->rhs_valid = true;
        c->steps += 1;
    }
    *bad = nullptr;
    return SPH_OK;
}

// The batched step as a captured graph (see sph_batch::graphs).  Returns
// false when the step must run launch by launch (*st stays SPH_OK) or on
// an error (*st, *bad set).
static bool batch_graph_step(sph_batch *b, const std::vector<sph_ctx *> &all,
                             const std::vector<sph_ctx *> &m32,
                             const std::vector<sph_ctx *> &m64, sph_status *st,
                             sph_ctx **bad) {
    *st = SPH_OK;
    if (!b->use_graphs || (uintptr_t)b->s <= 2) return false;
    std::vector<uintptr_t> comp{(uintptr_t)b->s, all.size()};
    for (sph_ctx *c : all) {
        comp.push_back((uintptr_t)c);
        comp.push_back((uintptr_t)c->cfg_version);
        comp.push_back((uintptr_t)c->anchor_version);
        comp.push_back((uintptr_t)c->n);
    }
    if (comp != b->comp) {
        b->comp = comp;
        b->same_comp = 0;
    }
    if (++b->same_comp <= 2) return false;
    for (sph_ctx *c : all) {
        if (!c->use_graphs || c->timing) return false;
        if ((uintptr_t)c->s <= 2 && c->s != b->s) return false;
        if (c->stage_want > c->stage_w) return false;
        // each build's list size known with headroom (no read-back)
        const bool sk = is_mixed(c);
        const uint32_t lt = sk ? c->last_total_skin : c->last_total;
        const int ltn = sk ? c->last_total_skin_n : c->last_total_n;
        const int n = c->n;
        if (!(lt > 0 && (size_t)lt * 2 <= c->list_cap && (long long)n * 10 <= (long long)ltn * 11 &&
              (long long)n * 10 >= (long long)ltn * 9))
            return false;
        if (!sk && !(c->last_total_n > 0)) return false;
    }
    for (sph_ctx *c : all) ensure_set_pk(c, &c->wall);
    std::vector<uintptr_t> key{(uintptr_t)b->s};
    for (sph_ctx *c : all) {
        const std::vector<uintptr_t> kc = graph_key(c);
        key.push_back((uintptr_t)c);
        key.insert(key.end(), kc.begin(), kc.end());
    }
    sph_batch::Graph *g = nullptr;
    for (auto &gg : b->graphs)
        if (gg.exec && gg.key == key) g = &gg;
    const size_t k = all.size();
    if (!g) {
        sph_batch::Graph *slot = &b->graphs[0];
        for (auto &gg : b->graphs)
            if (!gg.exec) {
                slot = &gg;
                break;
            }
        if (slot->exec) {
            slot = &b->graphs[b->graph_next_drop];
            b->graph_next_drop ^= 1;
        }
        if (slot->exec) cudaGraphExecDestroy(slot->exec);
        slot->exec = nullptr;
        slot->key.clear();
        if (!slot->d) {
            if (cudaMalloc(&slot->d, b->region) != cudaSuccess ||
                cudaMallocHost(&slot->h, b->region) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(slot->d);
                slot->d = nullptr;
                b->use_graphs = false;
                return false;
            }
        }
        // the slot's regions may still be read by its last replay
        if (cudaStreamSynchronize(b->s) != cudaSuccess) {
            *st = cuda_check(all[0], "sph_batch_step");
            *bad = all[0];
            return false;
        }
        struct Saved {
            double *f[NF], *falt[NF];
            int64_t *id, *id_alt;
            uint32_t tmask;
            float skin;
            long long steps;
            bool gv, rv;
            int launches;
        };
        std::vector<Saved> sv(k);
        for (size_t q = 0; q < k; ++q) {
            sph_ctx *c = all[q];
            memcpy(sv[q].f, c->f, sizeof(c->f));
            memcpy(sv[q].falt, c->falt, sizeof(c->falt));
            sv[q].id = c->id;
            sv[q].id_alt = c->id_alt;
            sv[q].tmask = c->tmask;
            sv[q].skin = c->skin;
            sv[q].steps = c->steps;
            sv[q].gv = c->grid_valid;
            sv[q].rv = c->rhs_valid;
            sv[q].launches = c->launches;
        }
        const long long bl0 = b->launches;
        Stager sg;
        sg.h = slot->h;
        sg.d = slot->d;
        sg.cap = b->region;
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ex = nullptr;
        sph_ctx *bad2 = nullptr;
        sph_status s2 = SPH_ECUDA;
        cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s2 = batch_body(b, all, m32, m64, sg, &bad2, true);
            e = cudaStreamEndCapture(b->s, &gr);
        }
        if (s2 == SPH_OK && e == cudaSuccess && gr) e = cudaGraphInstantiate(&ex, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (s2 != SPH_OK || e != cudaSuccess || !ex) {
            // undo the host side; the step runs launch by launch
            cudaGetLastError();
            if (ex) cudaGraphExecDestroy(ex);
            for (size_t q = 0; q < k; ++q) {
                sph_ctx *c = all[q];
                memcpy(c->f, sv[q].f, sizeof(c->f));
                memcpy(c->falt, sv[q].falt, sizeof(c->falt));
                c->id = sv[q].id;
                c->id_alt = sv[q].id_alt;
                c->tmask = sv[q].tmask;
                c->skin = sv[q].skin;
                c->steps = sv[q].steps;
                c->grid_valid = sv[q].gv;
                c->rhs_valid = sv[q].rv;
                c->launches = sv[q].launches;
                c->err.clear();
            }
            b->launches = bl0;
            b->use_graphs = false;
            return false;
        }
        slot->exec = ex;
        slot->key = key;
        slot->inst.assign(k, sph_batch::Inst());
        for (size_t q = 0; q < k; ++q) {
            sph_ctx *c = all[q];
            sph_batch::Inst &in = slot->inst[q];
            memcpy(in.f_after, c->f, sizeof(c->f));
            memcpy(in.falt_after, c->falt, sizeof(c->falt));
            in.id_after = c->id;
            in.id_alt_after = c->id_alt;
            in.tmask = c->tmask;
            in.skin = c->skin;
            in.launches = c->launches - sv[q].launches;
        }
        slot->launches = b->launches - bl0;
        g = slot;
    } else {
        for (size_t q = 0; q < k; ++q) {
            sph_ctx *c = all[q];
            const sph_batch::Inst &in = g->inst[q];
            memcpy(c->f, in.f_after, sizeof(c->f));
            memcpy(c->falt, in.falt_after, sizeof(c->falt));
            c->id = in.id_after;
            c->id_alt = in.id_alt_after;
            c->tmask = in.tmask;
            c->skin = in.skin;
            c->launches += in.launches;
            c->grid_valid = false;
            c->rhs_valid = true;
            c->steps += 1;
        }
        b->launches += g->launches;
    }
    // work queued on the contexts' streams before this call comes first
    join_from(b, all);
    if (cudaGraphLaunch(g->exec, b->s) != cudaSuccess) {
        *st = cuda_check(all[0], "sph_batch_step graph");
        *bad = all[0];
    }
    b->graph_steps += 1;
    return true;
}

extern "C" {

void sph_default_params(sph_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->lo[0] = p->lo[1] = 0.0;
    p->hi[0] = p->hi[1] = 1.0;
    p->rho0 = 1.0;
    p->cs = 10.0;
    p->nu = 0.0;
    p->U_ref = 1.0;
    p->hdx = 1.0;
    p->alpha_e = 1.5;
    p->split_alpha = 0.9;
    p->split_eps = 0.4;
    p->Cr = 1.08;
    p->merge_iters = 3;
    p->shift_iters = 3;
    p->precision = SPH_FP64;
    p->capacity = 0;
    p->pavg_mode = 0;
    p->edac_diff_denominator = 1;
    p->edac_rho_factor = 1;
    p->cell_c0 = 0.0;
    p->bg_Nr = 48.0;
    p->bg_smooth_iters = 3;
    p->vort_k = 0.0;
    p->n_bg = 0;
    p->bg_capacity = 0;
    p->sponge_width = 0.0;
}

sph_status sph_create(const sph_params *p, void *stream, sph_ctx **out) {
    if (out) *out = nullptr;
    if (!p || !out) {
        g_create_error = "sph_create: NULL argument";
        return SPH_EINVAL;
    }
    std::string why;
    if (p->dim != 2) why = "dim must be 2";
    else if (!(p->hi[0] > p->lo[0]) || !(p->hi[1] > p->lo[1])) why = "empty domain box";
    else if (p->capacity <= 0 || p->capacity > (1ll << 30)) why = "capacity must be in 1..2^30";
    else if (!(p->rho0 > 0) || !(p->cs > 0) || !(p->hdx > 0)) why = "rho0, cs, hdx must be positive";
    else if (!(p->nu >= 0)) why = "nu must be >= 0";
    else if (!(p->U_ref >= 0)) why = "U_ref must be >= 0";
    else if (p->precision != SPH_FP64 && p->precision != SPH_MIXED) why = "bad precision";
    else if (p->pavg_mode < 0 || p->pavg_mode > 1) why = "bad pavg_mode";
    else if (p->n_bg < 0 || p->bg_smooth_iters < 0) why = "n_bg, bg_smooth_iters must be >= 0";
    else if (p->bg_capacity > (1ll << 30)) why = "bg_capacity must be at most 2^30";
    if (!why.empty()) {
        g_create_error = "sph_create: " + why;
        return SPH_EINVAL;
    }
    std::string why2;
    sph_status st = new_ctx(p, (cudaStream_t)stream, false, out, &why2);
    if (st != SPH_OK) g_create_error = "sph_create: " + why2;
    else g_live_ctx.fetch_add(1);
    return st;
}

sph_status sph_load_particles(sph_ctx *c, sph_kind kind, long long n,
                              const sph_particles *src) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (n < 0 || (n > 0 && !src)) return fail(c, SPH_EINVAL, "sph_load_particles: bad n or src");
    if (kind == SPH_BACKGROUND) return load_background(c, n, src);
    if (kind == SPH_WALL) return load_walls(c, n, src);
    if (kind == SPH_REGION) {
        if (n > 0 && (!src->x || !src->y || !src->h))
            return fail(c, SPH_EINVAL, "sph_load_particles: region markers need x, y, h");
        return build_set(c, &c->region, n, n ? src->x : nullptr,
                         n ? src->y : nullptr, n ? src->h : nullptr, nullptr, 0,
                         nullptr);
    }
    if (kind != SPH_FLUID)
        return fail(c, SPH_EINVAL, "sph_load_particles: unknown kind");
    if (n > c->cap) return fail(c, SPH_ECAPACITY, "sph_load_particles: n exceeds capacity");
    if (n > 0 && (!src->x || !src->y || !src->m || !src->h))
        return fail(c, SPH_EINVAL, "sph_load_particles: x, y, m, h are required");
    double hmin = INFINITY;
    for (long long i = 0; i < n; ++i) {
        double h = src->h[i], m = src->m[i];
        if (!(h > 0) || !isfinite(h) || !(m > 0) || !isfinite(m))
            return fail(c, SPH_EINVAL, "sph_load_particles: h and m must be positive and finite");
        hmin = std::min(hmin, h);
        for (int a = 0; a < 2; ++a) {
            double q = a == 0 ? src->x[i] : src->y[i];
            bool in = c->dom.periodic[a] ? (q >= c->dom.lo[a] && q < c->dom.hi[a])
                                         : (q >= c->dom.lo[a] && q <= c->dom.hi[a]);
            if (!in || !isfinite(q))
                return fail(c, SPH_EINVAL, "sph_load_particles: position outside the box");
        }
    }
    double hmax = 0.0;
    for (long long i = 0; i < n; ++i) hmax = std::max(hmax, src->h[i]);
    sph_status gst = setup_fluid_grid(c, n, hmin, hmax);
    if (gst != SPH_OK) return gst;
    c->n = (int)n;
    // a new state: a non-finite rate or skin overrun reported for the old
    // one no longer applies
    cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->s);
    cudaMemsetAsync(c->d_skin_err, 0, sizeof(int), c->s);

    std::vector<double> tmp;
    auto put = [&](double *dst, const double *s, double dflt) {
        if (n == 0) return;
        if (s) {
            cudaMemcpyAsync(dst, s, sizeof(double) * n, cudaMemcpyHostToDevice, c->s);
        } else {
            tmp.assign((size_t)n, dflt);
            cudaMemcpyAsync(dst, tmp.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->s);
            cudaStreamSynchronize(c->s);
        }
    };
    put(c->f[F_X], src ? src->x : nullptr, 0);
    put(c->f[F_Y], src ? src->y : nullptr, 0);
    put(c->f[F_U], src ? src->u : nullptr, 0);
    put(c->f[F_V], src ? src->v : nullptr, 0);
    put(c->f[F_P], src ? src->p : nullptr, 0);
    put(c->f[F_RHO], src ? src->rho : nullptr, c->prm.rho0);
    put(c->f[F_M], src ? src->m : nullptr, 0);
    put(c->f[F_H], src ? src->h : nullptr, 0);
    put(c->f[F_MMIN], src ? src->mmin : nullptr, 0);
    put(c->f[F_MMAX], src ? src->mmax : nullptr, 0);
    if (c->f[F_DS]) put(c->f[F_DS], src ? src->ds : nullptr, c->prm.ds_max);
    c->next_id = n;
    if (n > 0 && src->id) {
        long long mx = -1;
        for (long long i = 0; i < n; ++i) mx = std::max<long long>(mx, src->id[i]);
        c->next_id = mx + 1;
    }
    if (n > 0) {
        if (src->id) {
            cudaMemcpyAsync(c->id, src->id, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->s);
        } else {
            std::vector<int64_t> ids((size_t)n);
            for (long long i = 0; i < n; ++i) ids[i] = i;
            cudaMemcpyAsync(c->id, ids.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->s);
            cudaStreamSynchronize(c->s);
        }
    }
    cudaStreamSynchronize(c->s);
    c->grid_valid = c->rhs_valid = c->have_dt = false;
    return cuda_check(c, "sph_load_particles");
}

sph_status sph_rhs(sph_ctx *c) {
    if (!c) return SPH_EINVAL;
    c->err.clear();
    if (c->n <= 0) return fail(c, SPH_ESTATE, "sph_rhs: no fluid particles loaded");
    compute_dt(c, nullptr, 0);
    sph_status st = rebuild(c, false);
    if (st != SPH_OK) return st;
    run_passes(c);
    store_rho(c);
    c->rhs_valid = true;
    return cuda_check(c, "sph_rhs");
}

sph_status sph_forces(sph_ctx *c, double *per_wall, double *total) {
    if (!c) return SPH_EINVAL;
    c->err.clear();
    if (!total) return fail(c, SPH_EINVAL, "sph_forces: total is NULL");
    for (int k = 0; k < 4; ++k) total[k] = 0.0;
    if (c->n <= 0) return fail(c, SPH_ESTATE, "sph_forces: no fluid particles loaded");
    const int nw = c->wall.n;
    if (nw <= 0) return SPH_OK;
    if (c->force_cap < nw) {
        cudaFree(c->d_force);
        c->d_force = nullptr;
        c->force_cap = 0;
        if (!dalloc(&c->d_force, (size_t)8 * nw + 4)) {
            cudaGetLastError();
            return fail(c, SPH_ENOMEM, "sph_forces: device allocation failed");
        }
        c->force_cap = nw;
    }
    // the wall condition and pass A at the current state
    compute_dt(c, nullptr, 0);
    sph_status st = rebuild(c, false);
    if (st != SPH_OK) return st;
    run_passes(c);
    c->rhs_valid = true;
    if (is_mixed(c))
        forces_launch<float>(c);
    else
        forces_launch<double>(c);
    double *out = c->d_force + 4 * (size_t)nw, *tot = c->d_force + 8 * (size_t)nw;
    launch_forces_total(c->s, nw, c->d_force, c->wall.id, out, tot);
    c->launches += 2;
    cudaMemcpyAsync(total, tot, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    if (per_wall)
        cudaMemcpyAsync(per_wall, out, 4 * sizeof(double) * nw,
                        cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_forces");
    return cuda_check(c, "sph_forces");
}

sph_status sph_force_coefficients(sph_ctx *c, double U, double L, double *out) {
    if (!c) return SPH_EINVAL;
    c->err.clear();
    if (!out) return fail(c, SPH_EINVAL, "sph_force_coefficients: out is NULL");
    if (!(U > 0) || !(L > 0) || !isfinite(U) || !isfinite(L))
        return fail(c, SPH_EINVAL, "sph_force_coefficients: U and L must be positive");
    double tot[4];
    sph_status st = sph_forces(c, nullptr, tot);
    if (st != SPH_OK) return st;
    // Eq. cdcl: force over the dynamic pressure times the length
    const double q = 0.5 * c->prm.rho0 * U * U * L;
    out[0] = tot[0] / q;
    out[1] = tot[2] / q;
    out[2] = tot[1] / q;
    return SPH_OK;
}

sph_status sph_step(sph_ctx *c, int nsteps, double *t_out) {
    if (!c) return SPH_EINVAL;
    c->err.clear();
    if (nsteps < 0) return fail(c, SPH_EINVAL, "sph_step: nsteps < 0");
    if (c->n <= 0) return fail(c, SPH_ESTATE, "sph_step: no fluid particles loaded");
    for (int s = 0; s < nsteps; ++s) {
        sph_status st = SPH_OK;
        if (!graph_step(c, &st)) {
            if (st != SPH_OK) return st;
            if ((st = pec_step(c, s == 0)) != SPH_OK) return st;
        } else if (st != SPH_OK) {
            return st;
        }
    }
    sph_status st = cuda_check(c, "sph_step");
    if (st != SPH_OK) return st;
    if (t_out) {
        double t = 0;
        int bad = 0;
        cudaMemcpyAsync(&t, c->d_t, sizeof(double), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(&bad, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_step sync");
        *t_out = t;
        if ((st = check_overflow(c, "sph_step")) != SPH_OK) return st;
        if (bad) {
            cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->s);   // reported once
            return fail(c, SPH_ENONFINITE, "sph_step: non-finite rate");
        }
    }
    return SPH_OK;
}


sph_status sph_batch_create(int max_instances, void *stream, sph_batch **out) {
    if (!out) return SPH_EINVAL;
    *out = nullptr;
    if (max_instances < 1 || max_instances > (1 << 20)) return SPH_EINVAL;
    sph_batch *b = new (std::nothrow) sph_batch;
    if (!b) return SPH_ENOMEM;
    b->s = (cudaStream_t)stream;
    b->cap = max_instances;
    // offsets: at most 96 groups a call (phases x precisions x team sizes),
    // each k + 1 entries and 16 bytes of alignment
    b->region = (size_t)max_instances * batch_bytes_per_instance() +
                96 * (((size_t)max_instances + 1) * sizeof(int) + 32) + 4096;
    bool ok = cudaMalloc(&b->d_buf, 2 * b->region) == cudaSuccess &&
              cudaMallocHost(&b->h_buf, 2 * b->region) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done[1], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->pack_blocks = pack_batch_blocks_per_sm() * gpu_sms();
    if (!ok) {
        cudaGetLastError();
        sph_batch_destroy(b);
        return SPH_ENOMEM;
    }
    *out = b;
    return SPH_OK;
}

sph_status sph_batch_destroy(sph_batch *b) {
    if (!b) return SPH_EINVAL;
    if (b->s || b->used[0] || b->used[1]) cudaStreamSynchronize(b->s);
    cudaFree(b->d_buf);
    cudaFreeHost(b->h_buf);
    for (auto &g : b->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        cudaFree(g.d);
        cudaFreeHost(g.h);
    }
    for (auto e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->ev) cudaEventDestroy(b->ev);
    delete b;
    return SPH_OK;
}

long long sph_batch_launches(const sph_batch *b) { return b ? b->launches : -1; }

sph_status sph_batch_step(sph_batch *b, sph_ctx *const *ctx, int k, double *t_out,
                          int *failed) {
    if (failed) *failed = -1;
    if (!b || !ctx || k < 1 || k > b->cap) return SPH_EINVAL;
    std::vector<sph_ctx *> all(ctx, ctx + k), m32, m64;
    for (int q = 0; q < k; ++q) {
        sph_ctx *c = all[q];
        if (!c) return SPH_EINVAL;
        for (int r = 0; r < q; ++r)
            if (all[r] == c) {
                if (failed) *failed = q;
                return fail(c, SPH_EINVAL, "sph_batch_step: a context appears twice");
            }
        c->err.clear();
        if (c->n <= 0) {
            if (failed) *failed = q;
            return fail(c, SPH_ESTATE, "sph_batch_step: no fluid particles loaded");
        }
        (is_mixed(c) ? m32 : m64).push_back(c);
    }
    auto index_of = [&](sph_ctx *c) {
        for (int q = 0; q < k; ++q)
            if (all[q] == c) return q;
        return -1;
    };
    sph_ctx *bad = nullptr;
    sph_status st = SPH_OK;
    if (!batch_graph_step(b, all, m32, m64, &st, &bad)) {
        if (st == SPH_OK) {
            // staging region of this call: free once the call before last ended
            const int r = b->calls & 1;
            if (b->used[r] && cudaEventSynchronize(b->done[r]) != cudaSuccess) {
                if (failed) *failed = 0;
                return cuda_check(all[0], "sph_batch_step");
            }
            Stager sg;
            sg.h = b->h_buf + r * b->region;
            sg.d = b->d_buf + r * b->region;
            sg.cap = b->region;
            st = batch_body(b, all, m32, m64, sg, &bad, false);
            if (st == SPH_OK) {
                cudaEventRecord(b->done[r], b->s);
                b->used[r] = true;
                b->calls += 1;
            }
        }
    }
    if (st != SPH_OK) {
        if (failed) *failed = bad ? index_of(bad) : 0;
        return st;
    }
    fork_to(b, all);   // later work on each context's stream follows the step
    for (int q = 0; q < k; ++q) {
        sph_status s2 = cuda_check(all[q], "sph_batch_step");
        if (s2 != SPH_OK) {
            if (failed) *failed = q;
            return s2;
        }
    }
    if (!t_out) return SPH_OK;
    if (cudaStreamSynchronize(b->s) != cudaSuccess) return cuda_check(all[0], "sph_batch_step sync");
    for (int q = 0; q < k; ++q) {
        sph_ctx *c = all[q];
        double t = 0;
        int nf = 0;
        cudaMemcpyAsync(&t, c->d_t, sizeof(double), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(&nf, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        sph_status s2 = check_overflow(c, "sph_batch_step");   // synchronises c->s
        t_out[q] = t;
        if (s2 == SPH_OK && nf) {
            cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->s);   // reported once
            s2 = fail(c, SPH_ENONFINITE, "sph_batch_step: non-finite rate");
        }
        if (s2 != SPH_OK) {
            if (failed) *failed = q;
            return s2;
        }
    }
    return SPH_OK;
}

long long sph_batch_graph_steps(const sph_batch *b) { return b ? b->graph_steps : -1; }

sph_status sph_batch_set_graphs(sph_batch *b, int enable) {
    if (!b) return SPH_EINVAL;
    b->use_graphs = enable != 0;
    return SPH_OK;
}

sph_status sph_adapt(sph_ctx *c, sph_adapt_stats *out) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (c->n <= 0) return fail(c, SPH_ESTATE, "sph_adapt: no fluid particles loaded");
    if (c->prm.n_bg > 0 && c->bg.n > 0 && ++c->adapt_calls % c->prm.n_bg == 0) {
        sph_status bs = sph_background(c, 1, nullptr);
        if (bs != SPH_OK) return bs;
    }
    sph_adapt_stats z;
    memset(&z, 0, sizeof(z));
    z.n_before = c->n;
    sph_status st = SPH_OK;
    cudaEvent_t ev;
    t_begin(c, 4, &ev);
    c->launches += launch_mass_sum(c->s, c->n, c->f[F_M], c->d_mass_part, c->d_mass);
    // resolution from the background (section 3.3)
    ensure_set_pk(c, &c->wall);
    if (c->bg.n > 0) {
        ensure_set_pk(c, &c->bg);
        // fluid anchor data at the current positions (moved since the last
        // rebuild)
        launch_anchor_pack(c->s, c->n, c->f[F_X], c->f[F_Y], c->f[F_H],
                           c->dom.lo, c->anchor_A, c->an, c->pk);
        BgArgs a;
        a.n = c->n;
        a.d = c->dom;
        a.g = set_grid(c->bg);
        a.an = c->an;
        a.pk = c->pk;
        a.bpk = c->bg.pk;
        a.x = c->f[F_X];
        a.y = c->f[F_Y];
        a.h = c->f[F_H];
        a.mmin = c->f[F_MMIN];
        a.mmax = c->f[F_MMAX];
        a.nb = c->bg.n;
        a.bx = c->bg.x;
        a.by = c->bg.y;
        a.bh = c->bg.h;
        a.bds = c->bg.ex[0];
        a.bcmin = c->bg.cmin;
        a.bid = c->bg.id;
        a.rho0 = c->prm.rho0;
        a.queue = c->tmp_b;
        a.nqueue = c->d_aux;
        launch_bg_mref(c->s, a);
        c->launches += 2;
    } else {
        cudaMemsetAsync(c->d_aux, 0, sizeof(uint32_t), c->s);
    }
    // split pass (section 3.1)
    uint32_t count = 0;
    if ((st = split_pass(c, &count)) != SPH_OK) {
        t_end(c, 4, ev);
        return st;
    }
    z.n_split = count;
    // merge rounds (section 3.2).  One list build serves several rounds:
    // merged-away particles stay in place, marked dead, and the kept ones
    // are updated in place, so the lists of the build still cover every
    // later partner while each merged particle's h / 2 plus its move since
    // the build stays within 1.5 h at the build (partners lie within
    // (h_i + h_j) / 2, the lists reach 3 max(h_i, h_j) at the build); a
    // merge beyond that flags the lists stale and the next round rebuilds
    // after compacting.  A round that merges nothing ends the rounds: it
    // left the state as it found it.
    {
        bool lists_ok = false, first = false, dead = false;
        int n_alive = c->n;
        auto compact_dead = [&]() {
            CompactArgs ca;
            for (int k = 0; k < NSTATE; ++k) {
                ca.src[k] = c->f[k];
                ca.dst[k] = c->falt[k];
            }
            ca.isrc = c->id;
            ca.idst = c->id_alt;
            launch_compact(c->s, c->n, c->tmp_a, c->tmp_b, ca);
            c->launches += 1;
            for (int k = 0; k < NSTATE; ++k) std::swap(c->f[k], c->falt[k]);
            std::swap(c->id, c->id_alt);
            c->n = n_alive;
            c->grid_valid = false;
            dead = false;
        };
        int *stale = (int *)(c->d_aux + 1);
        for (int r = 0; r < c->prm.merge_iters; ++r) {
            if (!lists_ok) {
                if (dead) compact_dead();
                if ((st = rebuild(c, false, true, 1.0f, false)) != SPH_OK) return st;
                cudaMemsetAsync(stale, 0, sizeof(int), c->s);
                lists_ok = true;
                first = true;
            }
            MergeArgs a;
            a.n = c->n;
            a.d = c->dom;
            for (int k = 0; k < NSTATE; ++k) a.f[k] = c->f[k];
            a.id = c->id;
            a.off = c->off;
            a.list = c->list;
            a.closest = c->closest;
            a.alive = c->tmp_a;
            a.an = c->an;
            a.pk = c->pk;
            a.alive_in = first ? nullptr : c->tmp_a;
            a.h0 = c->mh0;
            a.dsum = c->mds;
            a.budget = 1.5f * c->skin * (1.0f - 1e-3f);
            a.stale = stale;
            a.pkw = c->pk;
            a.mq = c->mq;
            for (int ax = 0; ax < 2; ++ax) {
                a.lo[ax] = c->dom.lo[ax];
                a.Ad[ax] = c->anchor_A[ax];
                a.invAd[ax] = 1.0 / c->anchor_A[ax];
            }
            first = false;
            launch_merge(c->s, a);
            exclusive_scan(c->s, c->tmp_a, c->tmp_b, c->n, c->d_total, c->sc, &c->launches);
            c->launches += a.alive_in ? 2 : 3;
            uint32_t keep = 0;
            int is_stale = 0;
            cudaMemcpyAsync(&keep, c->d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
            cudaMemcpyAsync(&is_stale, stale, sizeof(int), cudaMemcpyDeviceToHost, c->s);
            if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_adapt merge");
            if ((int)keep == n_alive) break;
            z.n_merged += n_alive - (int)keep;
            n_alive = (int)keep;
            dead = true;
            c->grid_valid = false;
            if (is_stale) lists_ok = false;
        }
        if (dead) compact_dead();
    }
    // shift rounds with Taylor correction, then the h update (3.2, 3.4)
    // One list build serves every shift round and the h update: a round
    // moves a particle by at most 0.25 h (Eq. shift-limit), so after k
    // rounds a pair is at most k (h_i + h_j) / 4 <= k max(h) / 2 closer,
    // and lists with skin 1 + k / 6 still hold N(i).  The shift sums vanish
    // outside N(i) (kernel support); the h update counts members only.
    // (mixed path only: on the FP64 path the wider lists cost more FP64
    // pair work than the rebuilds they save)
    const int ns = c->prm.shift_iters;
    if (ns <= 4 && is_mixed(c)) {
        if ((st = rebuild(c, false, true, 1.0f + ns / 6.0f + 0.01f)) != SPH_OK) return st;
        for (int r = 0; r < ns; ++r) {
            if (r > 0) pack(c, false);
            launch_shift_round(c->s, shift_args(c), is_mixed(c));
            c->launches += 3;
        }
        if (ns > 0) pack(c, false);
        ShiftArgs ha = shift_args(c);
        ha.filter = 1;
        launch_h_update(c->s, ha, is_mixed(c));
    } else {
        for (int r = 0; r < ns; ++r) {
            if ((st = rebuild(c, false)) != SPH_OK) return st;
            launch_shift_round(c->s, shift_args(c), is_mixed(c));
            c->launches += 3;
        }
        if ((st = rebuild(c, false)) != SPH_OK) return st;
        launch_h_update(c->s, shift_args(c), is_mixed(c));
    }
    c->launches += 2;
    c->launches += launch_mass_sum(c->s, c->n, c->f[F_M], c->d_mass_part, c->d_mass + 1);
    t_end(c, 4, ev);
    c->grid_valid = false;   // h changed since the last rebuild
    c->rhs_valid = false;
    double mass[2] = {0, 0};
    uint32_t nfb = 0;
    cudaMemcpyAsync(mass, c->d_mass, sizeof(mass), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(&nfb, c->d_aux, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_adapt");
    if ((st = check_overflow(c, "sph_adapt")) != SPH_OK) return st;
    z.mass_before = mass[0];
    z.mass_after = mass[1];
    z.n_bg_nearest = nfb;
    z.n_after = c->n;
    if (out) *out = z;
    return cuda_check(c, "sph_adapt");
}

sph_status sph_background(sph_ctx *c, int iterations, sph_bg_stats *out) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (c->bg.n <= 0) return fail(c, SPH_ESTATE, "sph_background: no background particles loaded");
    const sph_params &P = c->prm;
    if (!(P.ds_min > 0) || !(P.ds_max >= P.ds_min) || !isfinite(P.ds_max) ||
        !(P.Cr > 1) || !isfinite(P.Cr) || !(P.bg_Nr > 0) || !isfinite(P.bg_Nr))
        return fail(c, SPH_EINVAL,
                    "sph_background: need 0 < ds_min <= ds_max, Cr > 1, bg_Nr > 0");
    if (iterations <= 0)
        iterations = 3 * (int)ceil(log(P.ds_max / P.ds_min) / log(P.Cr));
    sph_bg_stats z;
    memset(&z, 0, sizeof(z));
    z.n_before = c->bg.n;
    sph_status st = ensure_bgc(c);
    if (st != SPH_OK) return st;
    sph_ctx *b = c->bgc;
    cudaEvent_t ev;
    t_begin(c, 4, &ev);
    const bool vort = P.vort_k > 0 && c->n > 0;
    if (vort && (st = compute_vorticity(c)) != SPH_OK) {
        t_end(c, 4, ev);
        return st;
    }
    sph_status ist = SPH_OK;
    int it = 0;
    for (; it < iterations && ist == SPH_OK; ++it) ist = bg_iteration(c, b, vort, &z);
    std::string ierr = c->err;
    // the refined set replaces the background (also after a failed
    // iteration: the completed ones are kept)
    const double *src[5] = {b->f[F_X], b->f[F_Y], b->f[F_H], b->f[F_DS], b->f[F_M]};
    st = build_set_device(c, &c->bg, b->n, src, 2, b->id);
    t_end(c, 4, ev);
    if (st != SPH_OK) {
        c->bgc_valid = false;
        return st;
    }
    c->bg_next_id = b->next_id;
    if ((st = check_overflow(b, "sph_background")) != SPH_OK) return fail(c, st, b->err);
    uint32_t cnt[2] = {0, 0};
    cudaMemcpyAsync(cnt, b->d_aux, sizeof(cnt), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_background");
    z.n_marked = cnt[0];
    z.n_vort = cnt[1];
    z.n_after = c->bg.n;
    z.iterations = ist == SPH_OK ? it : it - 1;
    if (out) *out = z;
    if (ist != SPH_OK) return fail(c, ist, ierr);
    return cuda_check(c, "sph_background");
}

static sph_status read_R(sph_ctx *c, const void *src, double *dst, long long n) {
    if (is_mixed(c)) {
        std::vector<float> tmp((size_t)n);
        cudaMemcpyAsync(tmp.data(), src, sizeof(float) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        for (long long i = 0; i < n; ++i) dst[i] = tmp[i];
    } else {
        cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
    }
    return SPH_OK;
}

static sph_status read_field(sph_ctx *c, sph_field field, void *dst, long long cap,
                             long long *n_out);

sph_status sph_read(sph_ctx *c, sph_field field, void *dst, long long cap,
                    long long *n_out) {
    if (!c) return SPH_EINVAL;
    c->err.clear();
    const int f = (int)field;
    if (!(f & SPH_READ_BY_ID)) return read_field(c, field, dst, cap, n_out);
    // by id: the field and then the ids in the current order (a read that
    // rebuilds first re-sorts), rows placed by the rank of their id
    const sph_field base = (sph_field)(f & ~SPH_READ_BY_ID);
    size_t es = 8;
    if (base == SPH_F_NNB) {
        es = 4;
    } else if (!((base >= SPH_F_X && base <= SPH_F_CELLKEY) || base == SPH_F_OMEGA)) {
        return fail(c, SPH_EINVAL, "sph_read: SPH_READ_BY_ID needs a per-particle field");
    }
    const long long n = c->n;
    if (n_out) *n_out = n;
    if (cap < n) return fail(c, SPH_ECAPACITY, "sph_read: buffer too small");
    if (n == 0) return SPH_OK;
    std::vector<unsigned char> tmp((size_t)n * es);
    std::vector<int64_t> ids((size_t)n);
    sph_status st = read_field(c, base, tmp.data(), n, nullptr);
    if (st != SPH_OK) return st;
    if ((st = read_field(c, SPH_F_ID, ids.data(), n, nullptr)) != SPH_OK) return st;
    std::vector<uint32_t> order((size_t)n);
    for (long long i = 0; i < n; ++i) order[i] = (uint32_t)i;
    std::sort(order.begin(), order.end(),
              [&](uint32_t a, uint32_t b) { return ids[a] < ids[b]; });
    unsigned char *o = (unsigned char *)dst;
    for (long long r = 0; r < n; ++r) memcpy(o + r * es, tmp.data() + (size_t)order[r] * es, es);
    return SPH_OK;
}

static sph_status read_field(sph_ctx *c, sph_field field, void *dst, long long cap,
                             long long *n_out) {
    if (!dst && cap > 0) return fail(c, SPH_EINVAL, "sph_read: dst is NULL");
    const long long n = c->n;
    auto need = [&](long long k) -> sph_status {
        if (n_out) *n_out = k;
        if (cap < k) return fail(c, SPH_ECAPACITY, "sph_read: buffer too small");
        return SPH_OK;
    };
    sph_status st;
    switch (field) {
    case SPH_F_X: case SPH_F_Y: case SPH_F_U: case SPH_F_V: case SPH_F_P:
    case SPH_F_RHO: case SPH_F_M: case SPH_F_H: case SPH_F_MMIN:
    case SPH_F_MMAX: {
        static const int map[] = {F_X, F_Y, F_U, F_V, F_P, F_RHO, F_M, F_H, F_MMIN, F_MMAX};
        if ((st = need(n)) != SPH_OK) return st;
        cudaMemcpyAsync(dst, c->f[map[field]], sizeof(double) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    }
    case SPH_F_ID:
        if ((st = need(n)) != SPH_OK) return st;
        cudaMemcpyAsync(dst, c->id, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    case SPH_F_BETA: case SPH_F_PAVG: case SPH_F_DRX: case SPH_F_DRY:
    case SPH_F_DPDT: case SPH_F_DUDT: case SPH_F_DVDT: {
        if (!c->rhs_valid) return fail(c, SPH_ESTATE, "sph_read: no right-hand side at this state");
        if ((st = check_overflow(c, "sph_read")) != SPH_OK) return st;
        if ((st = need(n)) != SPH_OK) return st;
        const void *srcs[] = {c->beta, c->pavg, c->drx, c->dry, c->dpdt, c->dudt, c->dvdt};
        return read_R(c, srcs[field - SPH_F_BETA], (double *)dst, n);
    }
    case SPH_F_NNB:
        if (!c->rhs_valid) return fail(c, SPH_ESTATE, "sph_read: no right-hand side at this state");
        if ((st = need(n)) != SPH_OK) return st;
        cudaMemcpyAsync(dst, c->nnb, sizeof(int) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    case SPH_F_CELLKEY: {
        if (!c->grid_valid) {
            if ((st = rebuild(c, false)) != SPH_OK) return st;
        }
        if ((st = need(n)) != SPH_OK) return st;
        uint64_t *o = (uint64_t *)dst;
        cudaMemcpyAsync(o, c->skey, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        const int sh = 2 * c->mbits;
        const uint64_t mask = (sh >= 64) ? ~0ull : ((1ull << sh) - 1ull);
        for (long long i = 0; i < n; ++i) o[i] = ((o[i] >> sh) << 58) | (o[i] & mask);
        return SPH_OK;
    }
    case SPH_F_NEIGH_OFF: case SPH_F_NEIGH_ID: {
        if (n == 0) {
            if (field == SPH_F_NEIGH_OFF) {
                if ((st = need(1)) != SPH_OK) return st;
                ((int64_t *)dst)[0] = 0;
            } else if (n_out) {
                *n_out = 0;
            }
            return SPH_OK;
        }
        if (!c->grid_valid) {
            if ((st = rebuild(c, false)) != SPH_OK) return st;
        }
        std::vector<uint32_t> off((size_t)n + 1);
        int ovf = 0;
        cudaMemcpyAsync(off.data(), c->off, sizeof(uint32_t) * (n + 1), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(&ovf, c->d_overflow, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        if (ovf) {
            c->last_total = c->last_total_skin = 0;
            return fail(c, SPH_ECAPACITY, "sph_read: neighbour list overflow");
        }
        const uint32_t total = off[n];
        if (field == SPH_F_NEIGH_OFF) {
            if ((st = need(n + 1)) != SPH_OK) return st;
            int64_t *o = (int64_t *)dst;
            for (long long i = 0; i <= n; ++i) o[i] = off[i];
            return SPH_OK;
        }
        if ((st = need(total)) != SPH_OK) return st;
        int64_t *dev = nullptr;
        if (cudaMalloc((void **)&dev, sizeof(int64_t) * std::max<uint32_t>(total, 1)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SPH_ENOMEM, "sph_read: neighbour list allocation failed");
        }
        launch_nbr_ids(c->s, c->n, c->off, c->list, c->id, dev);
        c->launches += 1;
        cudaMemcpyAsync(dst, dev, sizeof(int64_t) * total, cudaMemcpyDeviceToHost, c->s);
        cudaError_t e = cudaStreamSynchronize(c->s);
        cudaFree(dev);
        if (e != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    }
    case SPH_F_OMEGA:
        if ((st = need(n)) != SPH_OK) return st;
        if (n > 0 && (st = compute_vorticity(c)) != SPH_OK) return st;
        cudaMemcpyAsync(dst, c->omega, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    case SPH_F_BG_X: case SPH_F_BG_Y: case SPH_F_BG_H: case SPH_F_BG_M:
    case SPH_F_BG_DS: case SPH_F_BG_ID: {
        const long long nb = c->bg.n;
        if (n_out) *n_out = nb;
        if (cap < nb) return fail(c, SPH_ECAPACITY, "sph_read: buffer too small");
        if (nb == 0) return SPH_OK;
        const void *srcs[] = {c->bg.x, c->bg.y, c->bg.h, c->bg.ex[1], c->bg.ex[0], c->bg.id};
        cudaMemcpyAsync(dst, srcs[field - SPH_F_BG_X], 8 * nb, cudaMemcpyDeviceToHost, c->s);
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_read");
        return SPH_OK;
    }
    default:
        return fail(c, SPH_EINVAL, "sph_read: unknown field");
    }
}

sph_status sph_get_info(sph_ctx *c, sph_info *out) {
    if (!c || !out) return SPH_EINVAL;
    memset(out, 0, sizeof(*out));
    out->n = c->n;
    out->n_bg = c->bg.n;
    out->n_wall = c->wall.n;
    out->n_region = c->region.n;
    out->graph_steps = c->graph_launches;
    double t = 0, dt = 0;
    cudaMemcpyAsync(&t, c->d_t, sizeof(double), cudaMemcpyDeviceToHost, c->s);
    if (c->have_dt) cudaMemcpyAsync(&dt, c->d_dt, sizeof(double), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_get_info");
    out->t = t;
    out->dt = dt;
    out->c0 = c->c0;
    out->levels = c->lmax + 1;
    out->steps = c->steps;
    out->launches = c->launches;
    out->next_id = c->next_id;
    return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx *c, const sph_tune *in) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (!in) return fail(c, SPH_EINVAL, "sph_set_tuning: in is NULL");
    auto team_ok = [](int t) { return t == 0 || t == 1 || t == 4 || t == 16 || t == 32; };
    if (!(in->walk >= 0 && in->walk <= 3) || !team_ok(in->team_a) || !team_ok(in->team_b) ||
        !(in->walls >= 0 && in->walls <= 2) ||
        !(in->cell_scale <= 0 || (in->cell_scale >= 0.5 && in->cell_scale <= 4.0)))
        return fail(c, SPH_EINVAL, "sph_set_tuning: walk 0-3, teams 0/1/4/16/32, walls 0-2, cell_scale <= 0 or in [0.5, 4]");
    const double scale = in->cell_scale > 0 ? in->cell_scale : 1.0;
    c->walk_choice = in->walk;
    c->team_a = in->team_a;
    c->team_b = in->team_b;
    c->use_graphs = in->no_graphs ? 0 : 1;
    if (c->wall_mode != in->walls) {
        c->wall_mode = in->walls;
        c->grid_valid = false;
        c->rhs_valid = false;
    }
    if (scale != c->c0_scale) {
        c->c0_scale = scale;
        if (c->n > 0) {
            std::vector<double> h((size_t)c->n);
            cudaMemcpyAsync(h.data(), c->f[F_H], sizeof(double) * c->n,
                            cudaMemcpyDeviceToHost, c->s);
            if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_set_tuning");
            const double hmin = *std::min_element(h.begin(), h.end());
            const double hmax = *std::max_element(h.begin(), h.end());
            sph_status st = setup_fluid_grid(c, c->n, hmin, hmax);
            if (st != SPH_OK) return st;
        }
        c->grid_valid = false;
        c->rhs_valid = false;
    }
    return SPH_OK;
}

sph_status sph_autotune(sph_ctx *c, sph_tune *out) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (c->n <= 0) return fail(c, SPH_ESTATE, "sph_autotune: no fluid particles loaded");
    const bool timing_was = c->timing;
    sph_tune cur;
    memset(&cur, 0, sizeof(cur));
    cur.cell_scale = c->c0_scale;
    cur.walk = c->walk_choice;
    cur.team_a = c->team_a;
    cur.team_b = c->team_b;
    cur.no_graphs = c->use_graphs ? 0 : 1;
    cur.walls = c->wall_mode;
    sph_tune res = cur;
    // mean ms per launch of families 0 (pass B), 1 (pass A), 2 (build), 5
    // (walk) over `reps` builds + right-hand sides, after one untimed
    sph_status st = SPH_OK;
    auto measure = [&](int reps, double fam_ms[NFAM]) -> sph_status {
        for (int r = 0; r <= reps; ++r) {
            c->timing = r > 0;
            if (r == 1) {
                t_collect(c);
                for (int f = 0; f < NFAM; ++f) c->tm.ms[f] = 0, c->tm.count[f] = 0;
            }
            compute_dt(c, nullptr, 0);
            c->grid_valid = false;
            sph_status s2 = rebuild(c, false);
            if (s2 != SPH_OK) return s2;
            run_passes(c);
        }
        if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_autotune");
        t_collect(c);
        for (int f = 0; f < NFAM; ++f)
            fam_ms[f] = c->tm.count[f] ? c->tm.ms[f] / c->tm.count[f] : 0.0;
        for (int f = 0; f < NFAM; ++f) c->tm.ms[f] = 0, c->tm.count[f] = 0;
        return SPH_OK;
    };
    const int reps = 3;
    double fm[NFAM];
    // 1. level-0 cell size
    const double scales[3] = {1.0, 1.25, 1.5};
    int best = -1;
    for (int k = 0; k < 3; ++k) {
        sph_tune t = cur;
        t.cell_scale = scales[k];
        if ((st = sph_set_tuning(c, &t)) != SPH_OK) break;
        if ((st = measure(reps, fm)) != SPH_OK) break;
        res.ms_cell[k] = fm[2] + fm[1] + fm[0];
        if (best < 0 || res.ms_cell[k] < res.ms_cell[best]) best = k;
    }
    if (st == SPH_OK) {
        cur.cell_scale = scales[best];
        st = sph_set_tuning(c, &cur);
    }
    // 2. list build
    if (st == SPH_OK) {
        best = -1;
        for (int w = 1; w <= 3 && st == SPH_OK; ++w) {
            c->walk_choice = w;
            if ((st = measure(reps, fm)) != SPH_OK) break;
            res.ms_walk[w - 1] = fm[5];
            if (best < 0 || fm[5] < res.ms_walk[best - 1]) best = w;
        }
        cur.walk = best;
        c->walk_choice = best;
    }
    // 3. pass teams (both passes measured in the same runs)
    if (st == SPH_OK) {
        const int teams[4] = {1, 4, 16, 32};
        int ba = -1, bb = -1;
        for (int k = 0; k < 4 && st == SPH_OK; ++k) {
            c->team_a = c->team_b = teams[k];
            if ((st = measure(reps, fm)) != SPH_OK) break;
            res.ms_team_a[k] = fm[1];
            res.ms_team_b[k] = fm[0];
            if (ba < 0 || fm[1] < res.ms_team_a[ba]) ba = k;
            if (bb < 0 || fm[0] < res.ms_team_b[bb]) bb = k;
        }
        if (st == SPH_OK) {
            cur.team_a = teams[ba];
            cur.team_b = teams[bb];
        }
        c->team_a = cur.team_a;
        c->team_b = cur.team_b;
    }
    // 4. walls seen from the fluid (cell walk or lists)
    if (st == SPH_OK && c->wall.n > 0) {
        int bw = -1;
        for (int m = 1; m <= 2 && st == SPH_OK; ++m) {
            c->wall_mode = m;
            if ((st = measure(reps, fm)) != SPH_OK) break;
            res.ms_walls[m - 1] = fm[2] + fm[1] + fm[0];
            if (bw < 0 || res.ms_walls[m - 1] < res.ms_walls[bw - 1]) bw = m;
        }
        cur.walls = bw > 0 ? bw : cur.walls;
        c->wall_mode = cur.walls;
    }
    c->timing = timing_was;
    if (st != SPH_OK) return st;
    // end as sph_rhs does, with the chosen configuration
    compute_dt(c, nullptr, 0);
    c->grid_valid = false;
    if ((st = rebuild(c, false)) != SPH_OK) return st;
    run_passes(c);
    store_rho(c);
    c->rhs_valid = true;
    res.cell_scale = cur.cell_scale;
    res.walk = cur.walk;
    res.team_a = cur.team_a;
    res.team_b = cur.team_b;
    res.walls = cur.walls;
    if (out) *out = res;
    return cuda_check(c, "sph_autotune");
}

sph_status sph_set_timing(sph_ctx *c, int enable) {
    if (!c) return SPH_EINVAL;
    c->timing = enable != 0;
    return SPH_OK;
}

sph_status sph_kernel_time(sph_ctx *c, int family, double *ms,
                           long long *launches, int reset) {
    if (!c || family < 0 || family >= NFAM) return SPH_EINVAL;
    t_collect(c);
    if (ms) *ms = c->tm.ms[family];
    if (launches) *launches = c->tm.count[family];
    if (reset) {
        c->tm.ms[family] = 0;
        c->tm.count[family] = 0;
    }
    return SPH_OK;
}

sph_status sph_destroy(sph_ctx *c) {
    if (!c) return SPH_EINVAL;
    cudaStreamSynchronize(c->s);
    free_ctx(c);
    delete c;
    g_live_ctx.fetch_sub(1);
    return SPH_OK;
}

const char *sph_last_error(const sph_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

}  // extern "C"

namespace sph {
void set_noctx_error(const char *why) { g_create_error = why ? why : ""; }
}  // namespace sph

extern "C" {

unsigned long long sph_debug_failures(void) {
    return debug_failures_keys_sort() + debug_failures_adapt() + debug_failures_lists() +
           debug_failures_pairs();
}

int sph_debug_build(void) {
#ifdef SPH_DEBUG
    return 1;
#else
    return 0;
#endif
}

}  // extern "C"
