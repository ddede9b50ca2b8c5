// Internal declarations shared by the library's CUDA translation units.
// Adaptive-resolution WCSPH (Muta & Ramachandran, arXiv 2107.01276) on
// sm_103a.  Nothing here is part of the public C ABI (include/sph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sph.h"
#include "batch.cuh"

namespace sph {

constexpr int MAX_LEVELS = 32;      // cell levels c0 * 2^l, l < MAX_LEVELS
constexpr int MAX_MORTON_BITS = 29; // per axis
constexpr double PI = 3.14159265358979323846;
// Point of inflection of the quintic spline in q (section 2.1).
constexpr double XI_INFLECTION = 0.759298480738450;

// ---------------------------------------------------------------- domain --
struct Domain {
    double lo[2], hi[2], L[2], half[2];
    int periodic[2];
};

// One level of the multi-level cell grid.
struct Level {
    double c;      // nominal cell side c0 * 2^l (>= 3h of its particles)
    double w[2];   // cell width per axis (L / count on periodic axes)
    int n[2];      // cell count per axis
    float cf;      // c in FP32
    float invw[2]; // 1 / w in FP32 (cell ranges of queries)
    float wf[2];   // w in FP32 (cell rectangles of queries)
    float invP[2]; // 1 / (n w) in FP32 (periodic images of cells)
};

// Device view of the cell structure built by a rebuild.  Particles are
// sorted by skey = level << (2*mbits) | morton(ix, iy); every occupied cell
// has one entry in an open-addressing hash table (key -> [start, end)).
struct Grid {
    const uint64_t *tkey;   // hash slots, EMPTY = ~0
    const uint32_t *tstart;
    const uint32_t *tend;
    uint32_t tmask;         // table size - 1 (power of two)
    uint32_t level_mask;    // bit l set if level l is occupied
    int mbits;              // morton bits per axis
    int nlev;               // levels in use (top level = nlev - 1)
    const int *bbox;        // per level: min ix, max ix, min iy, max iy
    const float *tmaxh;     // per table slot: largest h of the cell (rounded
                            // up to float), or NULL
    // Occupancy map (static sets; NULL for the fluid): per level, the
    // level's bounding box cut into OCC_N x OCC_N blocks of cells, one bit
    // per block holding a particle; a query whose cells cover no set bit
    // skips the level without looking up a cell.
    const uint32_t *occ;
    Level lev[MAX_LEVELS];
};

constexpr int OCC_N = 64;                       // blocks per axis
constexpr int OCC_WORDS = MAX_LEVELS * OCC_N * (OCC_N / 32);

__host__ __device__ inline uint32_t compact2(uint64_t v) {
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v >> 4)) & 0x00ff00ff00ff00ffull;
    v = (v | (v >> 8)) & 0x0000ffff0000ffffull;
    v = (v | (v >> 16)) & 0x00000000ffffffffull;
    return (uint32_t)v;
}

// Block of cell index c on an axis whose occupied cells span [b0, b1].
__host__ __device__ inline int occ_block(int c, int b0, int b1) {
    return (int)(((long long)(c - b0) * OCC_N) / ((long long)b1 - b0 + 1));
}

// Sets the occupancy bits of n keyed particles (map zeroed beforehand,
// bounding boxes final).
void launch_occupancy(cudaStream_t s, int n, const uint64_t *key, int lshift,
                      const int *bbox, uint32_t *occ, int *launches);

constexpr uint64_t EMPTY_KEY = ~0ull;

__host__ __device__ inline uint64_t spread2(uint64_t v) {
    v &= 0x1fffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

__host__ __device__ inline uint32_t hash_slot(uint64_t k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// Minimum-image separation component, FP64, no contraction.
__device__ __forceinline__ double min_image(const Domain &d, int a,
                                            double s) {
    if (d.periodic[a]) {
        if (s > d.half[a])
            s = __dsub_rn(s, d.L[a]);
        else if (s < -d.half[a])
            s = __dadd_rn(s, d.L[a]);
    }
    return s;
}

// Records the reason of a failed call made without a context for
// sph_last_error(NULL) on the calling thread.
void set_noctx_error(const char *why);

// Bounds-check failures counted by each translation unit's kernels since
// its last call (debug builds, debug_checks.cuh; 0 otherwise).
unsigned long long debug_failures_keys_sort();
unsigned long long debug_failures_adapt();
unsigned long long debug_failures_lists();
unsigned long long debug_failures_pairs();

// ------------------------------------------------------------- context --
struct DeviceState;  // defined in sph_api.cu

// Radix sort + scan scratch owned by the context.
struct SortScratch {
    uint64_t *key_alt = nullptr;
    uint32_t *val_alt = nullptr;
    uint32_t *counts = nullptr;   // 256 * tiles
    uint32_t *scan_tmp = nullptr; // recursive scan block sums
    size_t counts_cap = 0, scan_cap = 0;
};

// Launch helpers implemented in keys_sort.cu
// Cell widths and counts of every level (host, FP64; same expressions as
// the level definition in the keys kernel).
void compute_levels(const Domain &dom, double c0, Level *lev);
void launch_keys(cudaStream_t s, int n, const Domain &dom, double c0,
                 int lmax, int mbits, const Level *lev, const double *x,
                 const double *y, const double *h, uint64_t *skey,
                 uint32_t *perm, uint32_t *level_mask, int *bbox,
                 uint32_t *zero = nullptr,    // zero[i] = 0 for i < n
                 uint32_t *zero2 = nullptr, uint32_t *zero3 = nullptr);
// Stable LSD radix sort of (skey, perm) over the low `bits` bits.
void radix_sort(cudaStream_t s, int n, int bits, uint64_t *key,
                uint32_t *val, SortScratch &sc, int *launches);
// Exclusive scan of n uint32 values (in may equal out); *total_dev (if not
// NULL) receives the sum.
void exclusive_scan(cudaStream_t s, const uint32_t *in, uint32_t *out,
                    int n, uint32_t *total_dev, SortScratch &sc,
                    int *launches);
size_t scan_scratch_elems(size_t n);
// off[i] = exclusive scan of own[i] + rev[i], off[n] = total, rev zeroed,
// in one launch; false (nothing done) if n is too large for one block.
bool list_offsets_small(cudaStream_t s, const uint32_t *own, uint32_t *rev,
                        uint32_t *off, int n, int *launches);
// Tile-count entries radix_sort needs in SortScratch::counts for n keys.
size_t radix_counts_elems(size_t n);
// h, tmaxh (may be NULL): also record each cell's largest h.
void build_cell_table(cudaStream_t s, int n, const uint64_t *skey,
                      uint64_t *tkey, uint32_t *tstart, uint32_t *tend,
                      uint32_t tmask, int *launches,
                      const double *h = nullptr, float *tmaxh = nullptr);
// out[k][i] = in[k][perm[i]] for up to 16 double arrays and 2 int64 arrays.
struct GatherList {
    const double *src[16];
    double *dst[16];
    int nd;
    const int64_t *isrc[2];
    int64_t *idst[2];
    int ni;
};
void gather_by_perm(cudaStream_t s, int n, const uint32_t *perm,
                    const GatherList &g, int *launches);
// gather_by_perm fused with the insertion of each cell's start into the
// table (keys reset to EMPTY_KEY beforehand).
void gather_insert(cudaStream_t s, int n, const uint32_t *perm,
                   const GatherList &g, const uint64_t *skey, uint64_t *tkey,
                   uint32_t *tstart, uint32_t tmask, int *launches);
struct RebuildReset {
    int *bbox;
    uint32_t *level_mask;
    uint64_t *tkey;
    uint32_t tslots;
    uint32_t *zero[5];
};
void launch_rebuild_reset(cudaStream_t s, const RebuildReset &r, int *launches);
int rebuild_reset_blocks(uint32_t tslots);   // its grid

// Cell keys of one set (the keys kernel's arguments).
struct KeysArgs {
    Domain dom;
    double c0, inv_c0;
    int lmax, mbits;
    Level lev[MAX_LEVELS];
    double invw[MAX_LEVELS][2];   // 1 / w per level and axis (FP64)
};
struct KeysRec {
    int n;
    KeysArgs a;
    const double *x, *y, *h;
    uint64_t *skey;
    uint32_t *perm, *level_mask;
    int *bbox;
    uint32_t *zero, *zero2, *zero3;   // per-particle counters zeroed (may be NULL)
};
KeysRec make_keys_rec(int n, const Domain &dom, double c0, int lmax, int mbits,
                      const Level *lev, const double *x, const double *y,
                      const double *h, uint64_t *skey, uint32_t *perm,
                      uint32_t *level_mask, int *bbox, uint32_t *zero,
                      uint32_t *zero2, uint32_t *zero3);

// Batched builds of small sets (batched step): the single-block sort and
// scan, and the per-particle kernels of a build, each as one launch over
// the work items of several instances (BatchSpan; an item is one block of
// the instance's single-launch grid).
struct RadixSmallRec {
    int n, passes;
    uint64_t *ka;
    uint32_t *va;
    uint64_t *kb;
    uint32_t *vb;
};
struct GatherInsertRec {
    int n;
    const uint32_t *perm;
    GatherList g;
    const uint64_t *skey;
    uint64_t *tkey;
    uint32_t *tstart;
    uint32_t tmask;
};
struct ScanSmallRec {
    const uint32_t *in;
    uint32_t *rev, *out;
    int n;
    uint32_t *total_dev;
    int write_total_at_n;
};
int radix_small_max();           // largest set the single-block sort takes
bool radix_small_available();    // its shared-memory limit could be raised
int scan_small_max();            // largest set the single-block scan takes
void launch_rebuild_reset_batch(cudaStream_t s, const RebuildReset *args, const BatchSpan &sp);
void launch_keys_batch(cudaStream_t s, const KeysRec *args, const BatchSpan &sp);
// false (nothing launched) if the shared-memory limit cannot be raised
bool launch_radix_small_batch(cudaStream_t s, const RadixSmallRec *args, const BatchSpan &sp,
                              int max_n);
void launch_gather_insert_batch(cudaStream_t s, const GatherInsertRec *args, const BatchSpan &sp);
void launch_scan_small_batch(cudaStream_t s, const ScanSmallRec *args, const BatchSpan &sp);
// cmin[start of each cell] = min of v over the cell (sorted set).
void launch_cell_min(cudaStream_t s, int n, const uint64_t *skey,
                     const double *v, double *cmin, int *launches);

// End of the cell of sorted particle i, if i is its last particle: the
// cell's table slot receives i + 1 and, with tmaxh, the cell's largest h
// rounded up to float.
__device__ __forceinline__ void table_mark_end(int i, int n,
                                               const uint64_t *skey,
                                               const uint64_t *tkey,
                                               uint32_t *tend, uint32_t tmask,
                                               const double *h = nullptr,
                                               float *tmaxh = nullptr) {
    const uint64_t k = skey[i];
    if (i + 1 < n && skey[i + 1] == k) return;
    uint32_t slot = hash_slot(k, tmask);
    for (uint32_t it = 0; it <= tmask; ++it) {
        const uint64_t t = tkey[slot];
        if (t == k) {
            tend[slot] = (uint32_t)(i + 1);
            if (tmaxh) {
                double m = h[i];
                for (int j = i - 1; j >= 0 && skey[j] == k; --j) m = fmax(m, h[j]);
                tmaxh[slot] = __double2float_ru(m);
            }
            return;
        }
        if (t == EMPTY_KEY) return;
        slot = (slot + 1) & tmask;
    }
}

}  // namespace sph
