// Argument blocks of the packing kernel and the neighbour-list build.
#pragma once

#include "batch.cuh"
#include "neighbors.cuh"
#include "sph_internal.cuh"

namespace sph {

struct PackArgs {
    int n;
    int lshift;                 // 2 * mbits: level = skey >> lshift
    int mixed;
    const uint64_t *skey;
    const double *x, *y, *h, *m, *p, *u, *v;
    double lo[2], Ad[2];        // anchor origin and side (FP64)
    double invAd[2];            // 1 / Ad
    Anchor an;
    uint8_t *lev;
    float4 *pk;                 // {xl, yl, h, gx | gy << 16}
    float *mf, *pf, *uf, *vf;
    // cell table: the last particle of each cell records its end
    const uint64_t *tkey;
    uint32_t *tend;
    uint32_t tmask;
    float *tmaxh;               // per slot: the cell's largest h
};

struct ListArgs {
    int n;
    Grid g;
    Domain d;
    Anchor an;
    const double *x, *y, *h;
    const float4 *pk;
    const uint8_t *lev;
    const uint64_t *skey;       // sorted cell keys (cells are runs of equal keys)
    uint32_t *own;              // entries found by i itself
    uint32_t *rev;              // reverse-entry counters / cursors
    uint32_t *off;              // n + 1 offsets
    uint32_t *list;             // neighbour indices
    uint32_t cap;               // list capacity (entries)
    int *overflow;
    uint32_t *longq, *nlong;    // particles with long reverse segments
    uint32_t *stage;            // n x stage_w staging rows of own entries
    uint32_t stage_w;           // row width (entries)
    uint32_t *max_own;          // largest own-entry count of the build
    uint32_t *queue, *nqueue;   // particles whose own entries overflow a row
    uint32_t *qref;             // per queued particle: its chunk's reference
                                // particle | 2^31 when the chunk spans two
                                // cells (cell-tile walks)
    // skin >= 1: lists hold every pair with r_ij < skin * 3 max(h_i, h_j)
    // (a superset of N(i) for particles that move less than the skin
    // allows); 1: exactly N(i)
    float skin;
    // walk: 1 per-particle team walk, 2 cell tiles with 4-lane teams, 3
    // cell tiles with a lane per particle, 4 the same with neighbouring
    // cells of a level merged into one chunk while they hold at most 32
    // particles, anything else: by set size
    int walk;
};

void launch_pack(cudaStream_t s, const PackArgs &a);
// packing over the work items of several instances (batched step); blocks:
// the persistent grid (resident blocks per SM from the function below
// times the SMs)
void launch_pack_batch(cudaStream_t s, const PackArgs *args, const BatchSpan &sp,
                       int blocks);
int pack_batch_blocks_per_sm();

// Batched builds of small sets (batched step): the per-particle team walk,
// the placement, the queue walk and the segment sorts over the work items
// of several instances (one item: one block of the instance's
// single-launch grid; the queue walk and the long-segment sort take
// fill_queue_blocks() and sort_long_blocks(n) items an instance, which
// change no result).
struct SortSegRec {
    int n;
    const uint32_t *off, *own;
    uint32_t *list;
    uint32_t cap;
    uint32_t *longq, *nlong;
};
int list_walk_kind(const ListArgs &a);   // 1 team walk, 2 / 3 cell tiles
int list_place_team(int n);              // lanes per particle of the placement
int fill_queue_blocks();
int sort_long_blocks(int n);
void launch_list_gather_batch(cudaStream_t s, int team, const ListArgs *args, const BatchSpan &sp);
void launch_list_place_batch(cudaStream_t s, int team, const ListArgs *args, const BatchSpan &sp);
void launch_list_fill_queue_batch(cudaStream_t s, const ListArgs *args, const BatchSpan &sp);
void launch_list_sort_rev_batch(cudaStream_t s, const SortSegRec *args, const BatchSpan &sp);
void launch_list_sort_long_batch(cudaStream_t s, const SortSegRec *args, const BatchSpan &sp);
void launch_anchor_pack(cudaStream_t s, int n, const double *x,
                        const double *y, const double *h, const double *lo,
                        const double *A, const Anchor &an, float4 *pk);
// The walk (own entries staged, reverse entries counted), then the
// offsets (off has n + 1 entries; tot_tmp needs n + 1), then the fill;
// entries past a.cap are dropped and flag a.overflow.  Before the walk,
// rev[0..n) and the counters nqueue, max_own and nlong must be zero (the
// rebuild's reset and key kernels do that).
void launch_list_walk(cudaStream_t s, const ListArgs &a, int *launches);
void list_offsets(cudaStream_t s, const ListArgs &a, SortScratch &sc,
                  uint32_t *tot_tmp, int *launches);
// queue: launch the second walk for rows that overflowed (false when the
// caller knows none did).
void build_lists_fill(cudaStream_t s, ListArgs a, bool mixed, bool queue,
                      int *launches);
// Each segment [off[i], off[i+1]) of list in ascending order (short ones in
// registers, long ones queued in longq / *nlong, which must be zero, for a
// warp sort).
void sort_segments(cudaStream_t s, int n, const uint32_t *off, uint32_t *list,
                   uint32_t cap, uint32_t *longq, uint32_t *nlong,
                   int *launches);

}  // namespace sph
