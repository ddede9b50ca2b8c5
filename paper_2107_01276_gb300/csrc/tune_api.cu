// Launch configuration of a context: sph_set_tuning and the autotuner
// (C ABI, include/sph.h).
#include "api.cuh"

extern "C" {

sph_status sph_set_tuning(sph_ctx *c, const sph_tune *in) {
    if (!c) return SPH_EINVAL;
    c->cfg_version += 1;
    c->err.clear();
    if (!in) return fail(c, SPH_EINVAL, "sph_set_tuning: in is NULL");
    auto team_ok = [](int t) { return t == 0 || t == 1 || t == 4 || t == 16 || t == 32; };
    if (!(in->walk >= 0 && in->walk <= 4) || !team_ok(in->team_a) || !team_ok(in->team_b) ||
        !(in->walls >= 0 && in->walls <= 2) ||
        !(in->cell_scale <= 0 || (in->cell_scale >= 0.5 && in->cell_scale <= 4.0)))
        return fail(c, SPH_EINVAL, "sph_set_tuning: walk 0-4, teams 0/1/4/16/32, walls 0-2, cell_scale <= 0 or in [0.5, 4]");
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
        // the team walk, the 4-lane cell tiles, the merged cell tiles
        const int walks[3] = {1, 2, 4};
        for (int q = 0; q < 3 && st == SPH_OK; ++q) {
            c->walk_choice = walks[q];
            if ((st = measure(reps, fm)) != SPH_OK) break;
            res.ms_walk[q] = fm[5];
            if (best < 0 || fm[5] < res.ms_walk[best]) best = q;
        }
        cur.walk = walks[best < 0 ? 0 : best];
        c->walk_choice = cur.walk;
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

}  // extern "C"
