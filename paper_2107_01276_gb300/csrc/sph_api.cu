// Host orchestration and C ABI (include/sph.h) of the GB300 adaptive WCSPH
// library.  Everything numerical is enqueued on the context's stream as
// the library's own kernels; the host only validates, sizes launches and
// moves buffers.
#include <mutex>

#include "api.cuh"

namespace {

// reason of the calling thread's last failed call made without a context
// (sph_create, sph_cell_sort_noalloc): sph_last_error(NULL)
thread_local std::string g_create_error;
static std::atomic<int> g_live_ctx{0};   // contexts made by sph_create, not yet destroyed


}  // namespace

static void free_set(StaticSet *S, cudaStream_t st) {
    void *ps[] = {S->occ, S->x, S->y, S->h, S->ex[0], S->ex[1], S->ex[2], S->id, S->pk, S->cmin,
                  S->key, S->tkey, S->perm, S->tstart, S->tend, S->tmaxh, S->bbox,
                  S->mask, S->sc.key_alt, S->sc.val_alt, S->sc.counts,
                  S->sc.scan_tmp};
    for (void *p : ps) dfree(p, st);
    *S = StaticSet();
}

namespace sph {
namespace api {

// ------------------------------------------------------------- helpers --
sph_status fail(sph_ctx *c, sph_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

sph_status cuda_check(sph_ctx *c, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(c, SPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return SPH_OK;
}



void t_begin(sph_ctx *c, int fam, cudaEvent_t *ev) {
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

void t_end(sph_ctx *c, int fam, cudaEvent_t ev0) {
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

void t_collect(sph_ctx *c) {
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

int bits_for(long long v) {   // bits to represent 0..v
    int b = 0;
    while ((1ll << b) <= v) ++b;
    return b;
}

Grid make_grid(const sph_ctx *c) {
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
Grid grid_for_kernels(const sph_ctx *c) {
    Grid g = make_grid(c);
    g.level_mask = (c->lmax >= 31) ? 0xffffffffu : ((1u << (c->lmax + 1)) - 1u);
    return g;
}

// ---------------------------------------------------------- the rebuild --
// Keys, stable sort, gather of the state in sorted order, cell table and
// (mixed path) float mirrors.  mid_step: also carry the PEC stage-start
// copies x0..p0.
ListArgs list_args(sph_ctx *c) {
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
    la.qref = c->lqref;
    la.nqueue = c->d_nlq;
    return la;
}

// Per-particle anchor records (and the mixed path's float mirrors) at the
// current positions; with table_end also the cell ends of the table (part
// of a rebuild).
PackArgs pack_args(sph_ctx *c, bool table_end) {
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
void pack(sph_ctx *c, bool table_end) {
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
bool want_wall_lists(const sph_ctx *c) {
    if (c->wall.n <= 0 || !c->wlist) return false;
    if (c->wall_mode == 1) return false;
    if (c->wall_mode == 2) return true;
    return c->wall.n >= 2048;
}

sph_status rebuild(sph_ctx *c, bool mid_step, bool exact,
                   float skin, bool for_walls) {
    const int n = c->n;
    const bool sk = skin > 1.0f;
    const uint32_t lt = sk ? c->last_total_skin : c->last_total;
    const int ltn = sk ? c->last_total_skin_n : c->last_total_n;
    if (exact && lt > 0 && (size_t)lt * 2 <= c->list_cap &&
        (long long)n * 10 <= (long long)ltn * 11 &&
        (long long)n * 10 >= (long long)ltn * 9)
        exact = false;
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->s, &capturing);
    if (c->stage_want > c->stage_w && capturing == cudaStreamCaptureStatusNone) {
        uint32_t *ns = nullptr;
        if (dalloc(&ns, (size_t)c->cap * c->stage_want, c->s)) {
            dfree(c->stage, c->s);   // after the last build's use of it, in stream order
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
            dfree(c->wlist, c->s);
            c->wlist = nullptr;
            c->wcap = 0;
            if (!dalloc(&c->wlist, want, c->s)) {
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
            dfree(c->list, c->s);
            c->list = nullptr;
            if (!dalloc(&c->list, want, c->s)) {
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

WallBcArgs wall_bc_args(sph_ctx *c) {
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

void run_passes(sph_ctx *c) {
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
static void pec(sph_ctx *c, double f) {
    const PecArgs<R> a = pec_args<R>(c, f);
    cudaEvent_t ev;
    t_begin(c, 3, &ev);
    launch_pec<R>(c->s, a);
    t_end(c, 3, ev);
    c->launches += 1;
}

void run_pec(sph_ctx *c, double f) {
    if (is_mixed(c))
        pec<float>(c, f);
    else
        pec<double>(c, f);
}

// Latest summation density into the FP64 state (density is recomputed,
// never integrated).
void store_rho(sph_ctx *c) {
    if (is_mixed(c)) {
        launch_float_to_double(c->s, c->n, (const float *)c->rhoR, c->f[F_RHO]);
        c->launches += 1;
    } else {
        cudaMemcpyAsync(c->f[F_RHO], c->rhoR, sizeof(double) * c->n,
                        cudaMemcpyDeviceToDevice, c->s);
    }
}

void compute_dt(sph_ctx *c, double *tacc, int nsteps) {
    c->launches += launch_dt(c->s, c->n, c->f[F_H], c->d_hmin, c->prm.U_ref, c->prm.cs,
              c->prm.nu, c->d_dt, tacc, nsteps);
    c->have_dt = true;
}

// Pinned host words of the contexts, 16 per context, carved from blocks
// kept for the life of the process: freeing page-locked memory would
// synchronise the device under every other context's work.
static std::mutex g_pin_mu;
static std::vector<uint32_t *> g_pin_free;

uint32_t *pinned_words_get() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int SLOTS = 256;
        uint32_t *blk = nullptr;
        if (cudaMallocHost((void **)&blk, SLOTS * 16 * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int k = SLOTS - 1; k >= 0; --k) g_pin_free.push_back(blk + 16 * k);
    }
    uint32_t *p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_words_put(uint32_t *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

void free_ctx(sph_ctx *c) {
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < NF; ++k) {
        dfree(c->f[k], c->s);
        dfree(c->falt[k], c->s);
    }
    void *ps[] = {c->nbA, c->nbB, c->id, c->id_alt, c->rhoR, c->beta, c->pavg, c->drx,
                  c->dry, c->V, c->rb2, c->dpdt, c->dudt, c->dvdt, c->mf,
                  c->pf, c->uf, c->vf, c->nnb, c->skey, c->perm,
                  c->sc.key_alt, c->sc.val_alt, c->sc.counts, c->sc.scan_tmp,
                  c->tkey, c->tstart, c->tend, c->tmaxh, c->bbox, c->level_mask,
                  c->cnt_tmp, c->d_dt, c->d_t, c->d_hmin, c->d_nonfinite,
                  c->d_total, c->lvl, c->pk, c->own, c->rev, c->off, c->list,
                  c->d_overflow, c->d_skin_err, c->longq, c->d_nlong, c->stage, c->lqueue, c->lqref, c->d_max_own,
                  c->d_nlq, c->tmp_a, c->tmp_b,
                  c->closest, c->mh0, c->mds, c->mq, c->d_mass, c->d_mass_part, c->wp, c->wugx,
                  c->wugy, c->d_aux, c->d_load};
    for (void *p : ps) dfree(p, c->s);
    dfree(c->omega, c->s);
    dfree(c->d_force, c->s);
    dfree(c->wcnt, c->s);
    dfree(c->woff, c->s);
    dfree(c->wcur, c->s);
    dfree(c->wlist, c->s);
    dfree(c->wlongq, c->s);
    dfree(c->d_wnlong, c->s);
    dfree(c->d_wmax, c->s);
    dfree(c->d_minmax, c->s);
    pinned_words_put(c->h_pin);
    c->h_pin = nullptr;
    if (c->bgc) {
        free_ctx(c->bgc);
        delete c->bgc;
        c->bgc = nullptr;
    }
    free_set(&c->bg, c->s);
    free_set(&c->wall, c->s);
    free_set(&c->region, c->s);
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
        dfree(tmp, c->s);
        dfree(tid, c->s);
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
        free_set(S, c->s);
        size_t N = (size_t)n;
        bool ok = dalloc(&S->x, N, c->s) && dalloc(&S->y, N, c->s) && dalloc(&S->h, N, c->s) &&
                  dalloc(&S->id, N, c->s) && dalloc(&S->key, N, c->s) && dalloc(&S->perm, N, c->s) &&
                  dalloc(&S->pk, N, c->s) &&
                  dalloc(&S->bbox, MAX_LEVELS * 4, c->s) && dalloc(&S->mask, 1, c->s) &&
                  dalloc(&S->occ, OCC_WORDS, c->s) &&
                  dalloc(&S->sc.key_alt, N, c->s) && dalloc(&S->sc.val_alt, N, c->s);
        for (int k = 0; k < nex; ++k) ok = ok && dalloc(&S->ex[k], N, c->s);
        ok = ok && dalloc(&S->cmin, N, c->s);
        size_t tiles = (N + 2047) / 2048;
        S->sc.counts_cap = 256 * tiles;
        S->sc.scan_cap = scan_scratch_elems(S->sc.counts_cap);
        ok = ok && dalloc(&S->sc.counts, S->sc.counts_cap, c->s) &&
             dalloc(&S->sc.scan_tmp, S->sc.scan_cap, c->s);
        uint32_t t = 1;
        while (t < 2u * (uint32_t)N) t <<= 1;
        ok = ok && dalloc(&S->tkey, t, c->s) && dalloc(&S->tstart, t, c->s) && dalloc(&S->tend, t, c->s) &&
             dalloc(&S->tmaxh, t, c->s);
        if (!ok) {
            cudaGetLastError();
            free_set(S, c->s);
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
    if (!dalloc(&tmp, (size_t)nf * n, c->s) || !dalloc(&tid, (size_t)n, c->s)) {
        cudaGetLastError();
        dfree(tmp, c->s);
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
sph_status build_set_device(sph_ctx *c, StaticSet *S, long long n,
                                   const double *const *src, int nex,
                                   const int64_t *ids) {
    if (n == 0) {
        S->n = 0;
        return SPH_OK;
    }
    const int nf = 3 + nex;
    double *tmp = nullptr;
    int64_t *tid = nullptr;
    if (!dalloc(&tmp, (size_t)nf * n, c->s) || !dalloc(&tid, (size_t)n, c->s)) {
        cudaGetLastError();
        dfree(tmp, c->s);
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
        dfree(tmp, c->s);
        dfree(tid, c->s);
        return cuda_check(c, "build_set_device");
    }
    double hmin;
    memcpy(&hmin, &mm[0], sizeof(double));
    return build_set_sorted(c, S, n, hmin, nex, tmp, tid);
}

// Anchor data of a static set for the context's current anchor lattice.
void ensure_set_pk(sph_ctx *c, StaticSet *S) {
    if (S->n <= 0 || c->anchor_version == 0 || S->pk_version == c->anchor_version)
        return;
    launch_anchor_pack(c->s, S->n, S->x, S->y, S->h, c->dom.lo, c->anchor_A,
                       c->an, S->pk);
    c->launches += 1;
    S->pk_version = c->anchor_version;
}

bool wall_pk_stale(const sph_ctx *c) {
    return c->wall.n > 0 && c->anchor_version != 0 && c->wall.pk_version != c->anchor_version;
}

Grid set_grid(const StaticSet &S) {
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

WallView wall_view(const sph_ctx *c) {
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
    dfree(c->wp, c->s);
    dfree(c->wugx, c->s);
    dfree(c->wugy, c->s);
    c->wp = c->wugx = c->wugy = nullptr;
    dfree(c->wlist, c->s);
    c->wlist = nullptr;
    c->wcap = 0;
    const size_t wcap = std::max<size_t>(4096, 256 * (size_t)n);
    if (n > 0 && !(dalloc(&c->wp, n, c->s) && dalloc(&c->wugx, n, c->s) && dalloc(&c->wugy, n, c->s) &&
                   dalloc(&c->wlist, wcap, c->s))) {
        cudaGetLastError();
        c->wall.n = 0;
        return fail(c, SPH_ENOMEM, "wall allocation failed");
    }
    if (n > 0) c->wcap = (uint32_t)wcap;
    c->grid_valid = false;   // the fluid's wall lists must be rebuilt
    c->rhs_valid = false;
    return SPH_OK;
}

uint32_t read_u32(sph_ctx *c, const uint32_t *dev, sph_status *st) {
    uint32_t v = 0;
    cudaMemcpyAsync(&v, dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) *st = cuda_check(c, "sync");
    return v;
}

// Allocate a context for p->capacity particles (parameters already
// validated).  has_ds: the context holds a background under construction.
sph_status new_ctx(const sph_params *p, cudaStream_t stream, bool has_ds,
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
        if (k != F_DS || has_ds) ok = ok && dalloc(&c->f[k], N, c->s) && dalloc(&c->falt[k], N, c->s);
    ok = ok && dalloc(&c->omega, N, c->s) && dalloc(&c->d_wmax, 1, c->s) && dalloc(&c->d_minmax, 2, c->s);
    ok = ok && dalloc(&c->id, N, c->s) && dalloc(&c->id_alt, N, c->s);
    double **rs[] = {(double **)&c->rhoR, (double **)&c->beta, (double **)&c->pavg,
                     (double **)&c->drx, (double **)&c->dry, (double **)&c->V,
                     (double **)&c->rb2, (double **)&c->dpdt, (double **)&c->dudt,
                     (double **)&c->dvdt};
    for (auto pp : rs) ok = ok && dalloc(pp, N, c->s);
    ok = ok && dalloc((double4_32a **)&c->nbA, N, c->s) && dalloc((double4_32a **)&c->nbB, N, c->s);
    ok = ok && dalloc(&c->mf, N, c->s) && dalloc(&c->pf, N, c->s) && dalloc(&c->uf, N, c->s) &&
         dalloc(&c->vf, N, c->s) && dalloc(&c->nnb, N, c->s);
    ok = ok && dalloc(&c->skey, N, c->s) && dalloc(&c->perm, N, c->s) &&
         dalloc(&c->sc.key_alt, N, c->s) && dalloc(&c->sc.val_alt, N, c->s);
    size_t tiles = (N + 2047) / 2048;
    c->sc.counts_cap = 256 * tiles;
    c->sc.scan_cap = scan_scratch_elems(std::max(c->sc.counts_cap, N + 1));
    ok = ok && dalloc(&c->sc.counts, c->sc.counts_cap, c->s) &&
         dalloc(&c->sc.scan_tmp, c->sc.scan_cap, c->s);
    uint32_t t = 1;
    while (t < 2u * (uint32_t)N) t <<= 1;
    c->tcap = t;
    ok = ok && dalloc(&c->tkey, t, c->s) && dalloc(&c->tstart, t, c->s) && dalloc(&c->tend, t, c->s) &&
         dalloc(&c->tmaxh, t, c->s);
    ok = ok && dalloc(&c->bbox, MAX_LEVELS * 4, c->s) && dalloc(&c->level_mask, 1, c->s) &&
         dalloc(&c->cnt_tmp, N + 1, c->s);
    ok = ok && dalloc(&c->d_dt, 2, c->s) && dalloc(&c->d_t, 1, c->s) && dalloc(&c->d_hmin, 1, c->s) &&
         dalloc(&c->d_nonfinite, 1, c->s) && dalloc(&c->d_total, 1, c->s) &&
         dalloc(&c->d_skin_err, 1, c->s) &&
         dalloc(&c->d_overflow, 1, c->s);
    ok = ok && dalloc(&c->lvl, N, c->s) && dalloc(&c->pk, N, c->s) && dalloc(&c->own, N, c->s) &&
         dalloc(&c->rev, N, c->s) && dalloc(&c->off, N + 1, c->s) &&
         dalloc(&c->longq, N, c->s) && dalloc(&c->d_nlong, 1, c->s) &&
         dalloc(&c->stage, N * c->stage_w, c->s) && dalloc(&c->lqueue, N, c->s) && dalloc(&c->lqref, N, c->s) &&
         dalloc(&c->d_nlq, 1, c->s) && dalloc(&c->d_max_own, 1, c->s);
    ok = ok && dalloc(&c->tmp_a, N + 1, c->s) && dalloc(&c->tmp_b, N + 1, c->s) &&
         dalloc(&c->closest, N, c->s) && dalloc(&c->mh0, N, c->s) && dalloc(&c->mds, N, c->s) &&
         dalloc(&c->mq, N, c->s) &&
         dalloc(&c->wcnt, N + 1, c->s) && dalloc(&c->woff, N + 1, c->s) && dalloc(&c->wcur, N, c->s) &&
         dalloc(&c->wlongq, N, c->s) && dalloc(&c->d_wnlong, 1, c->s) &&
         dalloc(&c->d_mass, 2, c->s) &&
         dalloc(&c->d_mass_part, 256, c->s) && dalloc(&c->d_aux, 4, c->s) &&
         dalloc(&c->d_load, 1, c->s) &&
         (c->h_pin = pinned_words_get()) != nullptr;
    c->list_cap = std::min<size_t>(N * 48, 0xffffffffull);
    ok = ok && dalloc(&c->list, c->list_cap, c->s);
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
    // the stream-ordered buffers become usable on every stream
    if (cudaStreamSynchronize(c->s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
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
sph_status setup_fluid_grid(sph_ctx *c, long long n, double hmin,
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

// Reports (and clears) a neighbour-list overflow of a build that ran
// without its sizing synchronisation, and particles that outran the skin
// of a step's lists; synchronises.
sph_status check_overflow(sph_ctx *c, const char *who) {
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
sph_status pec_step(sph_ctx *c, bool exact) {
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

// Contexts made by sph_create and not yet destroyed.
int live_contexts() { return g_live_ctx.load(); }

}  // namespace api
}  // namespace sph

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
    // the set goes into the alternate buffers and is checked there on the
    // device; only a set that passes replaces the state
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
    put(c->falt[F_X], src ? src->x : nullptr, 0);
    put(c->falt[F_Y], src ? src->y : nullptr, 0);
    put(c->falt[F_U], src ? src->u : nullptr, 0);
    put(c->falt[F_V], src ? src->v : nullptr, 0);
    put(c->falt[F_P], src ? src->p : nullptr, 0);
    put(c->falt[F_RHO], src ? src->rho : nullptr, c->prm.rho0);
    put(c->falt[F_M], src ? src->m : nullptr, 0);
    put(c->falt[F_H], src ? src->h : nullptr, 0);
    put(c->falt[F_MMIN], src ? src->mmin : nullptr, 0);
    put(c->falt[F_MMAX], src ? src->mmax : nullptr, 0);
    if (c->f[F_DS]) put(c->falt[F_DS], src ? src->ds : nullptr, c->prm.ds_max);
    if (n > 0) {
        if (src->id) {
            cudaMemcpyAsync(c->id_alt, src->id, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->s);
        } else {
            std::vector<int64_t> ids((size_t)n);
            for (long long i = 0; i < n; ++i) ids[i] = i;
            cudaMemcpyAsync(c->id_alt, ids.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->s);
            cudaStreamSynchronize(c->s);
        }
    }
    launch_load_check(c->s, n, c->falt[F_X], c->falt[F_Y], c->falt[F_H], c->falt[F_M],
                      n > 0 && src->id ? c->id_alt : nullptr, c->dom, c->d_load);
    c->launches += n > 0 ? 1 : 0;
    LoadCheckOut chk;
    cudaMemcpyAsync(c->h_pin, c->d_load, sizeof(LoadCheckOut), cudaMemcpyDeviceToHost, c->s);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sph_load_particles");
    memcpy(&chk, c->h_pin, sizeof(chk));
    if (chk.bad & LOAD_BAD_HM)
        return fail(c, SPH_EINVAL, "sph_load_particles: h and m must be positive and finite");
    if (chk.bad & LOAD_BAD_POS)
        return fail(c, SPH_EINVAL, "sph_load_particles: position outside the box");
    double hmin = INFINITY, hmax = 0.0;
    if (n > 0) {
        memcpy(&hmin, &chk.hmin, sizeof(double));
        memcpy(&hmax, &chk.hmax, sizeof(double));
    }
    sph_status gst = setup_fluid_grid(c, n, hmin, hmax);
    if (gst != SPH_OK) return gst;
    for (int k = 0; k < NSTATE; ++k) std::swap(c->f[k], c->falt[k]);   // F_DS included
    std::swap(c->id, c->id_alt);
    c->n = (int)n;
    c->next_id = n > 0 && src->id ? chk.idmax + 1 : n;
    // a new state: a non-finite rate or skin overrun reported for the old
    // one no longer applies
    cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->s);
    cudaMemsetAsync(c->d_skin_err, 0, sizeof(int), c->s);
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
        dfree(c->d_force, c->s);
        c->d_force = nullptr;
        c->force_cap = 0;
        if (!dalloc(&c->d_force, (size_t)8 * nw + 4, c->s)) {
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
        if (!dalloc(&dev, std::max<uint32_t>(total, 1), c->s)) {
            cudaGetLastError();
            return fail(c, SPH_ENOMEM, "sph_read: neighbour list allocation failed");
        }
        launch_nbr_ids(c->s, c->n, c->off, c->list, c->id, dev);
        c->launches += 1;
        cudaMemcpyAsync(dst, dev, sizeof(int64_t) * total, cudaMemcpyDeviceToHost, c->s);
        cudaError_t e = cudaStreamSynchronize(c->s);
        dfree(dev, c->s);
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
    const cudaStream_t s = c->s;
    cudaStreamSynchronize(s);
    free_ctx(c);
    delete c;
    // the frees run in stream order; the pool hands the memory back to the
    // device at this synchronisation
    cudaStreamSynchronize(s);
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
