// Argument blocks and launchers of the adaptive-refinement kernels
// (adapt.cu).
#pragma once

#include "sph_internal.cuh"
#include "walls.cuh"

namespace sph {

// The FP64 state arrays, in the order the context stores them.  S_DS (the
// size of a background particle, section 3.3) exists only in a context
// that holds the background under construction; elsewhere it is NULL.
enum { S_X = 0, S_Y, S_U, S_V, S_P, S_RHO, S_M, S_H, S_MMIN, S_MMAX, S_DS, NSTATE };

struct BgArgs {
    int n;                      // fluid particles
    Domain d;
    Grid g;                     // cell structure of the background
    const double *x, *y, *h;    // fluid
    double *mmin, *mmax;
    int nb;
    const double *bx, *by, *bh, *bds;   // background, sorted by its keys
    const double *bcmin;        // per background cell (at its first
                                // particle): least ds of the cell
    const int64_t *bid;         // background load index
    Anchor an;
    const float4 *pk, *bpk;     // anchor data of fluid and background
    double rho0;
    uint32_t *queue, *nqueue;   // fluid particles with no background in range
};

struct SplitArgs {
    int n, count;               // particles before the split, parents
    Domain d;
    double *f[NSTATE];
    int64_t *id;
    const uint32_t *parent;     // parent slot by rank (id order)
    long long next_id;
    double alpha, eps;
};

struct MergeArgs {
    int n;
    Domain d;
    double *f[NSTATE];
    const int64_t *id;
    const uint32_t *off, *list;
    Anchor an;
    const float4 *pk;           // anchor data at the current positions
    int *closest;
    uint32_t *alive;
    // Rounds over one list build (merged-away particles stay in place,
    // marked dead, until the rounds end): alive_in NULL in the first round
    // after a build (all alive), else the alive flags of the last round.
    // A merged particle that moved D since the build and now has smoothing
    // length h keeps every later merge partner inside the lists while
    // h / 2 + D <= budget h0 (h0: its h at the build; budget 1.5 times the
    // lists' skin, less a margin); otherwise *stale is set and the next
    // round rebuilds.
    const uint32_t *alive_in;
    float *h0, *dsum;
    float budget;
    int *stale;
    float4 *pkw;                // anchor records, refreshed for merged particles
    double lo[2], Ad[2], invAd[2];
    // Per particle {m rounded down, m_max rounded up} in FP32, or
    // {+inf, -inf} for a particle that cannot merge (dead, m_max <= 0 or
    // m > m_max): written for every particle in the first round after a
    // build, refreshed by each round for the particles it changes.
    float2 *mq;
};

struct CompactArgs {
    const double *src[NSTATE];
    double *dst[NSTATE];
    const int64_t *isrc;
    int64_t *idst;
};

struct ShiftArgs {
    int n;
    Domain d;
    double *f[NSTATE];
    const uint32_t *off, *list;
    double rho0, hdx;
    // scratch of the pair-arithmetic type (double or float)
    void *rho, *drx, *dry, *du, *dv, *dp, *hnew;
    WallView w;                 // walls join the densities and the shift
    // mixed path: FP32 anchor coordinates and mirrors of m, u, v, p
    Anchor an;
    const float4 *pk;
    const float *mf, *uf, *vf, *pf;
    // 1: the lists are a superset of N(i) (built with a skin); the mean
    // mass of the h update then counts only members
    int filter;
};

void launch_bg_mref(cudaStream_t s, const BgArgs &a);
void launch_split_flag(cudaStream_t s, int n, const double *m,
                       const double *mmax, uint32_t *flag);
void launch_split_collect(cudaStream_t s, int n, const uint32_t *flag,
                          const uint32_t *pos, const int64_t *id,
                          uint64_t *key, uint32_t *val);
void launch_split_emit(cudaStream_t s, const SplitArgs &a);
void launch_merge(cudaStream_t s, const MergeArgs &a);
void launch_compact(cudaStream_t s, int n, const uint32_t *alive,
                    const uint32_t *pos, const CompactArgs &c);
void launch_shift_round(cudaStream_t s, const ShiftArgs &a, bool mixed);
void launch_h_update(cudaStream_t s, const ShiftArgs &a, bool mixed);
// Returns the number of kernels launched.
int launch_mass_sum(cudaStream_t s, int n, const double *m, double *part,
                     double *out);

}  // namespace sph
