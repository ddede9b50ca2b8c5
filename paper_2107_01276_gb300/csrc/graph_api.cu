// The step as a CUDA graph (sph_step, include/sph.h): capture of a step's
// launches and their replay while the configuration holds.
#include "api.cuh"

namespace sph {
namespace api {

// Everything a step's launches depend on besides the device data: the
// buffers (the step swaps them), sizes, list storage, the launch
// configuration and the version of the loaded sets.
std::vector<uintptr_t> graph_key(const sph_ctx *c) {
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

void drop_graph(sph_ctx::StepGraph &g) {
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
bool graph_step(sph_ctx *c, sph_status *st) {
    *st = SPH_OK;
    const uintptr_t sh = (uintptr_t)c->s;
    if (!c->use_graphs || c->timing || sh <= 2) return false;
    // only while this is the one context of the process: capturing and
    // instantiating a graph wait on other threads' allocations and
    // synchronisations (up to seconds under the serving loop's load)
    if (live_contexts() > 1) return false;
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

}  // namespace api
}  // namespace sph
