// Cell keys and stable key sort with no device allocation: the same
// kernels as the neighbour-structure rebuild (keys, LSD radix sort), with
// their scratch in a fixed, file-scope device array instead of
// context-owned buffers.  For callers that cannot allocate device memory
// themselves; see sph_cell_sort_noalloc in include/sph.h.
#include <math.h>

#include <algorithm>

#include "pair_passes.cuh"
#include "sph_internal.cuh"

using namespace sph;

namespace {

// Largest particle count the fixed scratch serves.
constexpr long long NOALLOC_MAX_N = 1 << 18;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// scratch layout (bytes): alternate keys, alternate values, radix tile
// counts, scan block sums, level bounding boxes, level mask
constexpr size_t SZ_KEY = align256(sizeof(uint64_t) * NOALLOC_MAX_N);
constexpr size_t SZ_VAL = align256(sizeof(uint32_t) * NOALLOC_MAX_N);
constexpr size_t N_COUNTS = 256 * ((NOALLOC_MAX_N + 2047) / 2048);
constexpr size_t SZ_COUNTS = align256(sizeof(uint32_t) * N_COUNTS);
constexpr size_t N_SCAN = 4096;
constexpr size_t SZ_SCAN = align256(sizeof(uint32_t) * N_SCAN);
constexpr size_t SZ_BBOX = align256(sizeof(int) * MAX_LEVELS * 4);
constexpr size_t SZ_MASK = 256;
constexpr size_t SCRATCH_BYTES =
    SZ_KEY + SZ_VAL + SZ_COUNTS + SZ_SCAN + SZ_BBOX + SZ_MASK;

// ~3.2 MB, held by every GPU that loads the library until process exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

__global__ void k_canonical_keys(int n, int lshift, uint64_t *key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = key[i];
    const uint64_t mask = (1ull << lshift) - 1ull;
    key[i] = ((k >> lshift) << 58) | (k & mask);
}

// Status, with its reason kept for sph_last_error(NULL) on this thread.
sph_status nf(sph_status st, const char *why) {
    set_noctx_error(why);
    return st;
}

}  // namespace

extern "C" {

sph_status sph_cell_sort_noalloc(const sph_params *p, long long n,
                                 const double *x, const double *y,
                                 const double *h, uint64_t *key_out,
                                 uint32_t *perm_out, void *stream) {
    if (!p) return nf(SPH_EINVAL, "sph_cell_sort_noalloc: params is NULL");
    if (n < 0) return nf(SPH_EINVAL, "sph_cell_sort_noalloc: n < 0");
    if (n > NOALLOC_MAX_N)
        return nf(SPH_EINVAL,
                  "sph_cell_sort_noalloc: n exceeds the fixed scratch limit of "
                  "262144 particles");
    if (n > 0 && (!x || !y || !h || !key_out || !perm_out))
        return nf(SPH_EINVAL, "sph_cell_sort_noalloc: NULL array");
    if (p->dim != 2 || !(p->hi[0] > p->lo[0]) || !(p->hi[1] > p->lo[1]))
        return nf(SPH_EINVAL, "sph_cell_sort_noalloc: bad domain");
    double c0 = p->cell_c0 > 0 ? p->cell_c0 : 3.0 * p->hdx * p->ds_min;
    if (!(c0 > 0) || !isfinite(c0))
        return nf(SPH_EINVAL,
                  "sph_cell_sort_noalloc: set cell_c0 or ds_min (level-0 cell side)");
    Domain dom;
    for (int a = 0; a < 2; ++a) {
        dom.lo[a] = p->lo[a];
        dom.hi[a] = p->hi[a];
        dom.L[a] = p->hi[a] - p->lo[a];
        dom.half[a] = 0.5 * dom.L[a];
        dom.periodic[a] = p->periodic[a] ? 1 : 0;
    }
    double Lmax = std::max(dom.L[0], dom.L[1]);
    int lmax = 0;
    while (ldexp(c0, lmax) < Lmax) ++lmax;
    if (lmax >= MAX_LEVELS)
        return nf(SPH_EINVAL, "sph_cell_sort_noalloc: too many cell levels");
    Level lev[MAX_LEVELS];
    compute_levels(dom, c0, lev);
    long long nmax = std::max(lev[0].n[0], lev[0].n[1]);
    if (nmax >= (1ll << MAX_MORTON_BITS))
        return nf(SPH_EINVAL, "sph_cell_sort_noalloc: level-0 grid too fine");
    int mbits = 1;
    while ((1ll << mbits) <= nmax - 1) ++mbits;
    int lbits = 0;
    while ((1ll << lbits) <= lmax) ++lbits;
    if (n == 0) return SPH_OK;

    // the array's address on the current device, looked up on every call
    // (a device reset or a new primary context may move it); the first
    // lookup on a device loads the module there
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return nf(SPH_ECUDA, "sph_cell_sort_noalloc: cudaGetSymbolAddress failed");
    }
    unsigned char *base = (unsigned char *)ptr;
    SortScratch sc;
    sc.key_alt = (uint64_t *)base;
    sc.val_alt = (uint32_t *)(base + SZ_KEY);
    sc.counts = (uint32_t *)(base + SZ_KEY + SZ_VAL);
    sc.scan_tmp = (uint32_t *)(base + SZ_KEY + SZ_VAL + SZ_COUNTS);
    sc.counts_cap = N_COUNTS;
    sc.scan_cap = N_SCAN;
    if (radix_counts_elems((size_t)n) > N_COUNTS ||
        scan_scratch_elems(radix_counts_elems((size_t)n)) > N_SCAN)
        return nf(SPH_EINVAL, "sph_cell_sort_noalloc: scratch layout too small");
    int *bbox = (int *)(base + SZ_KEY + SZ_VAL + SZ_COUNTS + SZ_SCAN);
    uint32_t *mask = (uint32_t *)(base + SZ_KEY + SZ_VAL + SZ_COUNTS + SZ_SCAN + SZ_BBOX);

    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    // bounding boxes and level mask start empty on every call
    launch_reset_bbox(s, bbox, mask);
    launch_keys(s, (int)n, dom, c0, lmax, mbits, lev, x, y, h, key_out,
                perm_out, mask, bbox);
    radix_sort(s, (int)n, 2 * mbits + lbits, key_out, perm_out, sc, &launches);
    k_canonical_keys<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, 2 * mbits,
                                                             key_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nf(SPH_ECUDA, "sph_cell_sort_noalloc: launch failed");
    set_noctx_error("");
    return SPH_OK;
}

}  // extern "C"
