// Adaptation (sections 3.1-3.4: resolution from the background, split,
// merge rounds, shift rounds, h update) and the background construction
// (section 3.3): C ABI sph_adapt and sph_background, include/sph.h.
#include "api.cuh"

namespace sph {
namespace api {

// Pinned host words of a context (its h_pin): the counts the adaptation
// phases read back without blocking in the copy.
enum { HP_SPLIT = 0, HP_KEEP = 1, HP_STALE = 2, HP_NFB = 3, HP_MASS = 4 };   // HP_MASS: 2 doubles

// Split pass (section 3.1), first half: flag m > m_max, scan; the parent
// count is queued into h_pin[HP_SPLIT].
static void split_issue(sph_ctx *c) {
    launch_split_flag(c->s, c->n, c->f[F_M], c->f[F_MMAX], c->tmp_a);
    exclusive_scan(c->s, c->tmp_a, c->tmp_b, c->n, c->d_total, c->sc, &c->launches);
    c->launches += 1;
    cudaMemcpyAsync(c->h_pin + HP_SPLIT, c->d_total, sizeof(uint32_t),
                    cudaMemcpyDeviceToHost, c->s);
}

// Second half, once the count has arrived: rank the parents by id, emit
// the children.
static sph_status split_apply(sph_ctx *c, uint32_t count) {
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
    return SPH_OK;
}

// The whole split pass with its synchronisation (the parent count).
static sph_status split_pass(sph_ctx *c, uint32_t *count_out) {
    *count_out = 0;
    split_issue(c);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return cuda_check(c, "sync");
    const uint32_t count = c->h_pin[HP_SPLIT];
    sph_status st = split_apply(c, count);
    if (st == SPH_OK) *count_out = count;
    return st;
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
// its own (the owner's precision, ds in F_DS), so the fluid's rebuild,
// split and shift machinery serves it unchanged.  It is loaded from the context's
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
sph_status compute_vorticity(sph_ctx *c) {
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
        launch_shift_round(b->s, shift_args(b), is_mixed(b));
        b->grid_valid = false;
        c->launches += 4;
    }
    return SPH_OK;
}

// ------------------------------------------------------------ adaptation --
static void adapt_stop(AdaptJob &j, sph_status st) {
    t_end(j.c, 4, j.ev);
    j.st = st;
    j.phase = AdaptJob::DONE;
}

// Merged-away particles out of the state (the scan of the last merge
// round gave each kept one its row).
static void compact_dead(AdaptJob &j) {
    sph_ctx *c = j.c;
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
    c->n = j.n_alive;
    c->grid_valid = false;
    j.dead = false;
}

// Phase 1: the background construction when due, the mass before, the
// resolution from the background (section 3.3), the split flags and
// their count.
static void adapt_begin(AdaptJob &j) {
    sph_ctx *c = j.c;
    c->cfg_version += 1;
    c->err.clear();
    memset(&j.z, 0, sizeof(j.z));
    j.phase = AdaptJob::DONE;
    if (c->n <= 0) {
        j.st = fail(c, SPH_ESTATE, "sph_adapt: no fluid particles loaded");
        return;
    }
    if (c->prm.n_bg > 0 && c->bg.n > 0 && ++c->adapt_calls % c->prm.n_bg == 0) {
        const sph_status bs = sph_background(c, 1, nullptr);
        if (bs != SPH_OK) {
            j.st = bs;
            return;
        }
    }
    j.z.n_before = c->n;
    t_begin(c, 4, &j.ev);
    c->launches += launch_mass_sum(c->s, c->n, c->f[F_M], c->d_mass_part, c->d_mass);
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
    split_issue(c);
    j.phase = AdaptJob::SPLIT;
}

// One merge round (section 3.2), issued: its survivors and the stale flag
// are queued into the pinned words.  One list build serves several
// rounds: merged-away particles stay in place, marked dead, and the kept
// ones are updated in place, so the lists of the build still cover every
// later partner while each merged particle's h / 2 plus its move since
// the build stays within 1.5 h at the build (partners lie within
// (h_i + h_j) / 2, the lists reach 3 max(h_i, h_j) at the build); a merge
// beyond that flags the lists stale and the next round rebuilds after
// compacting.
static void merge_issue(AdaptJob &j) {
    sph_ctx *c = j.c;
    int *stale = (int *)(c->d_aux + 1);
    if (!j.lists_ok) {
        if (j.dead) compact_dead(j);
        const sph_status st = rebuild(c, false, true, 1.0f, false);
        if (st != SPH_OK) {
            adapt_stop(j, st);
            return;
        }
        cudaMemsetAsync(stale, 0, sizeof(int), c->s);
        j.lists_ok = true;
        j.first = true;
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
    a.alive_in = j.first ? nullptr : c->tmp_a;
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
    j.first = false;
    launch_merge(c->s, a);
    exclusive_scan(c->s, c->tmp_a, c->tmp_b, c->n, c->d_total, c->sc, &c->launches);
    c->launches += a.alive_in ? 2 : 3;
    cudaMemcpyAsync(c->h_pin + HP_KEEP, c->d_total, sizeof(uint32_t),
                    cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(c->h_pin + HP_STALE, stale, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    j.phase = AdaptJob::MERGE;
}

// Shift rounds with Taylor correction, then the h update (3.2, 3.4), the
// mass after; the masses and the count of nearest-background fallbacks
// are queued into the pinned words.  One list build serves every shift
// round and the h update: a round moves a particle by at most 0.25 h
// (Eq. shift-limit), so after k rounds a pair is at most
// k (h_i + h_j) / 4 <= k max(h) / 2 closer, and lists with skin 1 + k / 6
// still hold N(i).  The shift sums vanish outside N(i) (kernel support);
// the h update counts members only.  (mixed path only: on the FP64 path
// the wider lists cost more FP64 pair work than the rebuilds they save)
static void finish_issue(AdaptJob &j) {
    sph_ctx *c = j.c;
    if (j.dead) compact_dead(j);
    sph_status st;
    const int ns = c->prm.shift_iters;
    if (ns <= 4 && is_mixed(c)) {
        if ((st = rebuild(c, false, true, 1.0f + ns / 6.0f + 0.01f)) != SPH_OK)
            return adapt_stop(j, st);
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
            if ((st = rebuild(c, false)) != SPH_OK) return adapt_stop(j, st);
            launch_shift_round(c->s, shift_args(c), is_mixed(c));
            c->launches += 3;
        }
        if ((st = rebuild(c, false)) != SPH_OK) return adapt_stop(j, st);
        launch_h_update(c->s, shift_args(c), is_mixed(c));
    }
    c->launches += 2;
    c->launches += launch_mass_sum(c->s, c->n, c->f[F_M], c->d_mass_part, c->d_mass + 1);
    t_end(c, 4, j.ev);
    c->grid_valid = false;   // h changed since the last rebuild
    c->rhs_valid = false;
    cudaMemcpyAsync(c->h_pin + HP_MASS, c->d_mass, 2 * sizeof(double),
                    cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(c->h_pin + HP_NFB, c->d_aux, sizeof(uint32_t),
                    cudaMemcpyDeviceToHost, c->s);
    j.phase = AdaptJob::FINISH;
}

// The next phase of j once its stream has been synchronised.
static void adapt_advance(AdaptJob &j) {
    sph_ctx *c = j.c;
    switch (j.phase) {
    case AdaptJob::SPLIT: {
        const uint32_t count = c->h_pin[HP_SPLIT];
        const sph_status st = split_apply(c, count);
        if (st != SPH_OK) return adapt_stop(j, st);
        j.z.n_split = count;
        j.lists_ok = j.first = j.dead = false;
        j.n_alive = c->n;
        j.round = 0;
        if (c->prm.merge_iters > 0)
            merge_issue(j);
        else
            finish_issue(j);
        return;
    }
    case AdaptJob::MERGE: {
        // a round that merges nothing ends the rounds: it left the state
        // as it found it
        const int keep = (int)c->h_pin[HP_KEEP];
        const int is_stale = (int)c->h_pin[HP_STALE];
        if (keep != j.n_alive) {
            j.z.n_merged += j.n_alive - keep;
            j.n_alive = keep;
            j.dead = true;
            c->grid_valid = false;
            if (is_stale) j.lists_ok = false;
            if (++j.round < c->prm.merge_iters) return merge_issue(j);
        }
        return finish_issue(j);
    }
    case AdaptJob::FINISH: {
        j.phase = AdaptJob::DONE;
        if ((j.st = check_overflow(c, "sph_adapt")) != SPH_OK) return;
        double mass[2];
        memcpy(mass, c->h_pin + HP_MASS, sizeof(mass));
        j.z.mass_before = mass[0];
        j.z.mass_after = mass[1];
        j.z.n_bg_nearest = c->h_pin[HP_NFB];
        j.z.n_after = c->n;
        j.st = cuda_check(c, "sph_adapt");
        return;
    }
    default:
        return;
    }
}

void adapt_run(AdaptJob *jobs, int k) {
    for (int i = 0; i < k; ++i) adapt_begin(jobs[i]);
    for (;;) {
        bool any = false;
        for (int i = 0; i < k; ++i) {
            AdaptJob &j = jobs[i];
            if (j.phase == AdaptJob::DONE) continue;
            if (cudaStreamSynchronize(j.c->s) != cudaSuccess) {
                if (j.phase != AdaptJob::FINISH) t_end(j.c, 4, j.ev);
                j.st = cuda_check(j.c, "sph_adapt");
                j.phase = AdaptJob::DONE;
                continue;
            }
            any = true;
        }
        if (!any) return;
        for (int i = 0; i < k; ++i)
            if (jobs[i].phase != AdaptJob::DONE) adapt_advance(jobs[i]);
    }
}

}  // namespace api
}  // namespace sph

extern "C" {

sph_status sph_adapt(sph_ctx *c, sph_adapt_stats *out) {
    if (!c) return SPH_EINVAL;
    AdaptJob j;
    j.c = c;
    adapt_run(&j, 1);
    if (j.st == SPH_OK && out) *out = j.z;
    return j.st;
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

}  // extern "C"
