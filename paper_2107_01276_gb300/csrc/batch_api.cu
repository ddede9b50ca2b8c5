// The batched step over several contexts (C ABI sph_batch_*), see
// include/sph.h.
#include <thread>

#include "api.cuh"

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

// body(a, e) over contiguous runs [a, e) of [0, k): one run per host
// thread, up to the host's hardware threads (the caller's among them),
// each thread on the caller's current device.
template <class F>
static void host_runs(int k, F body) {
    const int nt = std::min(k, std::max(1, (int)std::thread::hardware_concurrency()));
    if (nt <= 1) {
        body(0, k);
        return;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) {
        const int a = (int)((long long)k * t / nt);
        const int e = (int)((long long)k * (t + 1) / nt);
        th.emplace_back([&body, dev, a, e] {
            cudaSetDevice(dev);
            body(a, e);
        });
    }
    body(0, (int)((long long)k / nt));
    for (auto &x : th) x.join();
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
    // their builds issued from host threads (outside a capture, which
    // takes the launches of the capturing thread only)
    std::vector<sph_status> bst(rest.size(), SPH_OK);
    auto build_run = [&](int a, int e) {
        for (int q = a; q < e; ++q) {
            sph_ctx *c = rest[q];
            compute_dt(c, c->d_t, 1);
            if ((bst[q] = rebuild(c, false, true, is_mixed(c) ? 1.1f : 1.0f)) != SPH_OK) return;
        }
    };
    if (capturing)
        build_run(0, (int)rest.size());
    else
        host_runs((int)rest.size(), build_run);
    for (size_t q = 0; q < rest.size(); ++q)
        if (bst[q] != SPH_OK) {
            *bad = rest[q];
            join_from(b, rest);
            return bst[q];
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

sph_status sph_batch_adapt(sph_batch *b, sph_ctx *const *ctx, int k,
                           sph_adapt_stats *stats, sph_status *status) {
    if (!b || !ctx || k < 1 || k > b->cap) return SPH_EINVAL;
    for (int q = 0; q < k; ++q) {
        if (!ctx[q]) return SPH_EINVAL;
        for (int r = 0; r < q; ++r)
            if (ctx[r] == ctx[q])
                return fail(ctx[q], SPH_EINVAL, "sph_batch_adapt: a context appears twice");
    }
    std::vector<AdaptJob> jobs(k);
    for (int q = 0; q < k; ++q) jobs[q].c = ctx[q];
    // the host work (launches, read-backs) of the adaptations spread over
    // host threads, each adapting its run of contexts in lockstep
    host_runs(k, [&jobs](int a, int e) { adapt_run(jobs.data() + a, e - a); });
    sph_status first = SPH_OK;
    for (int q = 0; q < k; ++q) {
        if (status) status[q] = jobs[q].st;
        if (stats) {
            if (jobs[q].st == SPH_OK)
                stats[q] = jobs[q].z;
            else
                memset(&stats[q], 0, sizeof(stats[q]));
        }
        if (first == SPH_OK) first = jobs[q].st;
    }
    return first;
}

long long sph_batch_graph_steps(const sph_batch *b) { return b ? b->graph_steps : -1; }

sph_status sph_batch_set_graphs(sph_batch *b, int enable) {
    if (!b) return SPH_EINVAL;
    b->use_graphs = enable != 0;
    return SPH_OK;
}

}  // extern "C"
