// Cell keys, stable LSD radix sort, exclusive scan, permutation gather and
// the cell hash table: the neighbour-structure rebuild that the paper runs
// before every iteration (section 3.4, step iii: "update the nearest
// neighbor search").  All HBM-bound; no tensor cores.
#include <algorithm>

#include "batch.cuh"
#include "debug_checks.cuh"
#include "sph_internal.cuh"

namespace sph {

// ------------------------------------------------------------------ keys --
// Level l_i: smallest l >= 0 with c0 2^l >= t, t = (3 h_i) / c0 in FP64,
// capped at lmax.  Cell index floor((x - lo) / w_l) clamped to the level's
// cell count.  skey = l << (2 mbits) | morton(ix, iy), ix on even bits.
__device__ __forceinline__ int level_of(double h, double c0, int lmax) {
    double t = __ddiv_rn(__dmul_rn(3.0, h), c0);
    int l = 0;
    if (t > 1.0) {
        int e;
        double f = frexp(t, &e);
        l = (f == 0.5) ? e - 1 : e;
    }
    return l > lmax ? lmax : l;
}

__device__ __forceinline__ int cell_coord(double x, double lo, double w,
                                          int ncell) {
    double q = floor(__ddiv_rn(__dsub_rn(x, lo), w));
    int c;
    if (q < 0.0)
        c = 0;
    else if (q > (double)(ncell - 1))
        c = ncell - 1;
    else
        c = (int)q;
    return c;
}

// Fast forms of the two quotients above: the product with a rounded
// reciprocal is within 2^-51 relative of the correctly rounded quotient, so
// where it lies farther than 1e-12 (relative) from every integer (cell
// index) or power of two (level), it gives the same floor or exponent; the
// rare cases closer than that take the correctly rounded division.  GB300's
// FP64 division costs tens of FP64 operations at a small fraction of the
// FP32 rate; a product costs one.
__device__ __forceinline__ int level_of_fast(double h, double c0,
                                             double inv_c0, int lmax) {
    const double y = __dmul_rn(__dmul_rn(3.0, h), inv_c0);
    if (y < 1.0 - 1e-12) return 0;
    if (y > 1.0 + 1e-12) {
        int e;
        const double f = frexp(y, &e);
        if (f > 0.5 + 1e-12 && f < 1.0 - 1e-12) return e > lmax ? lmax : e;
    }
    return level_of(h, c0, lmax);
}

__device__ __forceinline__ int cell_coord_fast(double x, double lo, double w,
                                               double invw, int ncell) {
    const double t = __dsub_rn(x, lo);
    const double y = __dmul_rn(t, invw);
    const double fy = floor(y);
    const double tol = 1e-12 * fmax(1.0, fabs(y));
    if (!(y - fy > tol && fy + 1.0 - y > tol)) return cell_coord(x, lo, w, ncell);
    int c;
    if (fy < 0.0)
        c = 0;
    else if (fy > (double)(ncell - 1))
        c = ncell - 1;
    else
        c = (int)fy;
    return c;
}

__device__ __forceinline__ void keys_at(const KeysRec &r, int vb) {
    const int n = r.n;
    const KeysArgs &a = r.a;
    const double *__restrict__ x = r.x;
    const double *__restrict__ y = r.y;
    const double *__restrict__ h = r.h;
    uint64_t *__restrict__ skey = r.skey;
    uint32_t *__restrict__ perm = r.perm;
    uint32_t *level_mask = r.level_mask;
    int *bbox = r.bbox;
    uint32_t *__restrict__ zero = r.zero;
    uint32_t *__restrict__ zero2 = r.zero2;
    uint32_t *__restrict__ zero3 = r.zero3;
    __shared__ int sb[MAX_LEVELS * 4];
    __shared__ uint32_t smask;
    for (int t = threadIdx.x; t < MAX_LEVELS * 4; t += blockDim.x)
        sb[t] = (t & 1) ? -1 : 0x7fffffff;
    if (threadIdx.x == 0) smask = 0;
    __syncthreads();
    int i = vb * blockDim.x + threadIdx.x;
    if (i < n) {
        int l = level_of_fast(h[i], a.c0, a.inv_c0, a.lmax);
        const Level &L = a.lev[l];
        int ix = cell_coord_fast(x[i], a.dom.lo[0], L.w[0], a.invw[l][0], L.n[0]);
        int iy = cell_coord_fast(y[i], a.dom.lo[1], L.w[1], a.invw[l][1], L.n[1]);
        uint64_t m = spread2((uint64_t)ix) | (spread2((uint64_t)iy) << 1);
        skey[i] = ((uint64_t)l << (2 * a.mbits)) | m;
        perm[i] = (uint32_t)i;
        if (zero) zero[i] = 0;
        if (zero2) zero2[i] = 0;
        if (zero3) zero3[i] = 0;
        atomicOr(&smask, 1u << l);
        atomicMin(&sb[l * 4 + 0], ix);
        atomicMax(&sb[l * 4 + 1], ix);
        atomicMin(&sb[l * 4 + 2], iy);
        atomicMax(&sb[l * 4 + 3], iy);
    }
    __syncthreads();
    uint32_t msk = smask;
    for (int t = threadIdx.x; t < MAX_LEVELS * 4; t += blockDim.x) {
        int l = t >> 2;
        if (!(msk & (1u << l))) continue;
        if (t & 1)
            atomicMax(&bbox[t], sb[t]);
        else
            atomicMin(&bbox[t], sb[t]);
    }
    if (threadIdx.x == 0 && msk) atomicOr(level_mask, msk);
}

__global__ void k_keys(KeysRec r) { keys_at(r, blockIdx.x); }

void compute_levels(const Domain &dom, double c0, Level *lev) {
    for (int l = 0; l < MAX_LEVELS; ++l) {
        double c = ldexp(c0, l);
        lev[l].c = c;
        lev[l].cf = (float)c;
        for (int ax = 0; ax < 2; ++ax) {
            double Lx = dom.L[ax];
            long long nc;
            double w;
            if (dom.periodic[ax]) {
                nc = (long long)floor(Lx / c);
                if (nc < 1) nc = 1;
                w = Lx / (double)nc;
            } else {
                nc = (long long)ceil(Lx / c);
                if (nc < 1) nc = 1;
                w = c;
            }
            if (nc > (1ll << MAX_MORTON_BITS)) nc = 1ll << MAX_MORTON_BITS;
            lev[l].n[ax] = (int)nc;
            lev[l].w[ax] = w;
            lev[l].invw[ax] = (float)(1.0 / w);
            lev[l].wf[ax] = (float)w;
            lev[l].invP[ax] = (float)(1.0 / ((double)nc * w));
        }
    }
}

KeysRec make_keys_rec(int n, const Domain &dom, double c0, int lmax, int mbits,
                      const Level *lev, const double *x, const double *y,
                      const double *h, uint64_t *skey, uint32_t *perm,
                      uint32_t *level_mask, int *bbox, uint32_t *zero,
                      uint32_t *zero2, uint32_t *zero3) {
    KeysRec r;
    r.n = n;
    KeysArgs &a = r.a;
    a.dom = dom;
    a.c0 = c0;
    a.lmax = lmax;
    a.mbits = mbits;
    a.inv_c0 = 1.0 / c0;
    for (int l = 0; l < MAX_LEVELS; ++l) {
        a.lev[l] = lev[l];
        a.invw[l][0] = 1.0 / lev[l].w[0];
        a.invw[l][1] = 1.0 / lev[l].w[1];
    }
    r.x = x;
    r.y = y;
    r.h = h;
    r.skey = skey;
    r.perm = perm;
    r.level_mask = level_mask;
    r.bbox = bbox;
    r.zero = zero;
    r.zero2 = zero2;
    r.zero3 = zero3;
    return r;
}

void launch_keys(cudaStream_t s, int n, const Domain &dom, double c0,
                 int lmax, int mbits, const Level *lev, const double *x,
                 const double *y, const double *h, uint64_t *skey,
                 uint32_t *perm, uint32_t *level_mask, int *bbox,
                 uint32_t *zero, uint32_t *zero2, uint32_t *zero3) {
    if (n <= 0) return;
    const KeysRec r = make_keys_rec(n, dom, c0, lmax, mbits, lev, x, y, h, skey, perm,
                                    level_mask, bbox, zero, zero2, zero3);
    int bs = 256;
    k_keys<<<(n + bs - 1) / bs, bs, 0, s>>>(r);
}

// ------------------------------------------------------------ radix sort --
// 8-bit digits, 256 threads (8 warps) per tile of 8 * 32 * ITEMS keys.
// Warp w ranks its contiguous sub-tile step by step with __match_any_sync;
// the per-(warp, digit) running counts in shared memory make the rank
// stable.  Tile counts are scanned digit-major, so the scatter keeps the
// input order among equal digits across tiles as well.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

template <bool SCATTER>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix(int n, int shift, int ntiles, const uint64_t *__restrict__ kin,
            const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
            uint32_t *__restrict__ vout, uint32_t *__restrict__ counts) {
    __shared__ uint32_t cnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS)
        (&cnt[0][0])[t] = 0;
    __syncthreads();
    const int tile = blockIdx.x;
    const long long base = (long long)tile * RS_TILE + (long long)w * 32 * RS_ITEMS;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t rank[RS_ITEMS];
    uint64_t key[RS_ITEMS];
    int dig[RS_ITEMS];
#pragma unroll
    for (int s = 0; s < RS_ITEMS; ++s) {
        long long e = base + s * 32 + lane;
        bool ok = e < n;
        uint64_t k = ok ? kin[e] : 0;
        int d = ok ? (int)((k >> shift) & 255u) : 256;
        key[s] = k;
        dig[s] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (ok) before = cnt[w][d];
        __syncwarp();
        if (ok && lane == leader) cnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[s] = before + __popc(peers & lt);
    }
    __syncthreads();
    if (!SCATTER) {
        int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) tot += cnt[ww][d];
        counts[(size_t)d * ntiles + tile] = tot;
        return;
    }
    {
        int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < RS_ITEMS; ++s) {
        long long e = base + s * 32 + lane;
        if (e >= n) continue;
        int d = dig[s];
        uint32_t pos = counts[(size_t)d * ntiles + tile] + cnt[w][d] + rank[s];
        kout[pos] = key[s];
        vout[pos] = vin[e];
    }
}

// Small sets (n <= RSS_MAX): every pass in one block of 32 warps, keys
// and values staged in shared memory.  Warp w owns a contiguous chunk; the
// per-(warp, digit) counts, scanned digit-major, give each warp's scatter
// base, and the warp ranks its chunk 32 keys at a time with
// __match_any_sync, so the sort is stable exactly like the tiled form.
// Intermediate passes scatter into (kb, vb) and reload; the last pass
// scatters into (ka, va).
constexpr int RSS_THREADS = 1024;
constexpr int RSS_WARPS = RSS_THREADS / 32;
constexpr int RSS_MAX = 16384;

__device__ __forceinline__ void radix_small_at(int n, int passes, uint64_t *ka,
                                               uint32_t *va, uint64_t *kb,
                                               uint32_t *vb) {
    extern __shared__ uint64_t sk[];          // n keys, then n values
    uint32_t *sv = (uint32_t *)(sk + n);
    __shared__ uint32_t cnt[RSS_WARPS][256];
    __shared__ uint32_t dtot[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int chunk = (((n + RSS_WARPS - 1) / RSS_WARPS) + 31) & ~31;
    const int wb = w * chunk, we = min(n, wb + chunk);
    for (int e = threadIdx.x; e < n; e += RSS_THREADS) {
        sk[e] = ka[e];
        sv[e] = va[e];
    }
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const bool last = p == passes - 1;
        uint64_t *kout = last ? ka : kb;
        uint32_t *vout = last ? va : vb;
        for (int t = threadIdx.x; t < RSS_WARPS * 256; t += RSS_THREADS)
            (&cnt[0][0])[t] = 0;
        __syncthreads();
        for (int b = wb; b < we; b += 32) {
            const int e = b + lane;
            const bool ok = e < we;
            const int d = ok ? (int)((sk[e] >> shift) & 255u) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            uint32_t before = 0;
            if (ok) before = cnt[w][d];
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) cnt[w][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x < 256) {            // per digit: prefix over warps
            const int d = threadIdx.x;
            uint32_t run = 0;
            for (int ww = 0; ww < RSS_WARPS; ++ww) {
                const uint32_t c = cnt[ww][d];
                cnt[ww][d] = run;
                run += c;
            }
            dtot[d] = run;
        }
        __syncthreads();
        if (threadIdx.x < 32) {             // digit bases (exclusive scan of 256)
            uint32_t v[8], sum = 0;
            for (int k = 0; k < 8; ++k) {
                v[k] = dtot[lane * 8 + k];
                sum += v[k];
            }
            uint32_t x = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t pre = x - sum;
            for (int k = 0; k < 8; ++k) {
                dtot[lane * 8 + k] = pre;
                pre += v[k];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < RSS_WARPS * 256; t += RSS_THREADS)
            (&cnt[0][0])[t] += dtot[t & 255];
        __syncthreads();
        for (int b = wb; b < we; b += 32) {
            const int e = b + lane;
            const bool ok = e < we;
            uint64_t k = 0;
            int d = 256;
            if (ok) {
                k = sk[e];
                d = (int)((k >> shift) & 255u);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            uint32_t before = 0;
            if (ok) before = cnt[w][d];
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) cnt[w][d] = before + __popc(peers);
            __syncwarp();
            if (ok) {
                const uint32_t pos = before + __popc(peers & lt);
                kout[pos] = k;
                vout[pos] = sv[e];
            }
        }
        __syncthreads();
        if (!last) {
            for (int e = threadIdx.x; e < n; e += RSS_THREADS) {
                sk[e] = kb[e];
                sv[e] = vb[e];
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(RSS_THREADS)
    k_radix_small(int n, int passes, uint64_t *ka, uint32_t *va, uint64_t *kb,
                  uint32_t *vb) {
    radix_small_at(n, passes, ka, va, kb, vb);
}

// The dynamic shared-memory limit of k_radix_small, raised once per device.
static bool radix_small_ready() {
    static signed char ok[64];   // 0 unknown, 1 ready, -1 unavailable
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    if (ok[dev] == 0) {
        ok[dev] = cudaFuncSetAttribute(k_radix_small,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       RSS_MAX * 12) == cudaSuccess ? 1 : -1;
        if (ok[dev] < 0) cudaGetLastError();
    }
    return ok[dev] == 1;
}

size_t radix_counts_elems(size_t n) {
    return 256 * ((n + RS_TILE - 1) / RS_TILE);
}

void radix_sort(cudaStream_t s, int n, int bits, uint64_t *key,
                uint32_t *val, SortScratch &sc, int *launches) {
    if (n <= 1 || bits <= 0) return;
    if (n <= RSS_MAX && radix_small_ready()) {
        k_radix_small<<<1, RSS_THREADS, (size_t)n * 12, s>>>(
            n, (bits + 7) / 8, key, val, sc.key_alt, sc.val_alt);
        *launches += 1;
        return;
    }
    int ntiles = (n + RS_TILE - 1) / RS_TILE;
    uint64_t *ka = key, *kb = sc.key_alt;
    uint32_t *va = val, *vb = sc.val_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix<false><<<ntiles, RS_THREADS, 0, s>>>(n, shift, ntiles, ka, va,
                                                     kb, vb, sc.counts);
        exclusive_scan(s, sc.counts, sc.counts, 256 * ntiles, nullptr, sc,
                       launches);
        k_radix<true><<<ntiles, RS_THREADS, 0, s>>>(n, shift, ntiles, ka, va,
                                                    kb, vb, sc.counts);
        *launches += 2;
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != key) {
        cudaMemcpyAsync(key, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
}

// ------------------------------------------------------------------ scan --
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v,
                                                    uint32_t *total) {
    __shared__ uint32_t ws[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < SC_THREADS / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SC_THREADS / 32) ws[lane] = t;
    }
    __syncthreads();
    uint32_t pre = (w > 0 ? ws[w - 1] : 0) + x - v;
    if (total) *total = ws[SC_THREADS / 32 - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int n,
                              uint32_t *__restrict__ sums) {
    long long b0 = (long long)blockIdx.x * SC_TILE;
    uint32_t acc = 0;
    for (int s = 0; s < SC_ITEMS; ++s) {
        long long e = b0 + s * SC_THREADS + threadIdx.x;
        if (e < n) acc += in[e];
    }
    uint32_t tot;
    block_excl_scan(acc, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, int n,
                            const uint32_t *__restrict__ offs,
                            uint32_t *total_dev) {
    long long b0 = (long long)blockIdx.x * SC_TILE +
                   (long long)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t acc = 0;
#pragma unroll
    for (int s = 0; s < SC_ITEMS; ++s) {
        long long e = b0 + s;
        v[s] = e < n ? in[e] : 0;
        acc += v[s];
    }
    uint32_t tot;
    uint32_t pre = block_excl_scan(acc, &tot);
    pre += offs ? offs[blockIdx.x] : 0;
#pragma unroll
    for (int s = 0; s < SC_ITEMS; ++s) {
        long long e = b0 + s;
        if (e < n) out[e] = pre;
        pre += v[s];
    }
    if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == SC_THREADS - 1)
        *total_dev = pre;
}

size_t scan_scratch_elems(size_t n) {
    size_t tot = 0;
    while (n > (size_t)SC_TILE) {
        n = (n + SC_TILE - 1) / SC_TILE;
        tot += n;
    }
    return tot + 1;
}

static void scan_rec(cudaStream_t s, const uint32_t *in, uint32_t *out, int n,
                     uint32_t *total_dev, uint32_t *tmp, int *launches) {
    int nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb <= 1) {
        k_scan_down<<<1, SC_THREADS, 0, s>>>(in, out, n, nullptr, total_dev);
        *launches += 1;
        return;
    }
    uint32_t *sums = tmp;
    k_scan_reduce<<<nb, SC_THREADS, 0, s>>>(in, n, sums);
    scan_rec(s, sums, sums, nb, nullptr, tmp + nb, launches);
    k_scan_down<<<nb, SC_THREADS, 0, s>>>(in, out, n, sums, total_dev);
    *launches += 2;
}

// Small scans (n <= 1024 * 32): one block of 1024 threads, thread t owns
// a contiguous chunk; two passes over the chunk (sum, then write), so in
// may equal out.  With `rev`, the values are in[i] + rev[i] and rev is
// zeroed (the neighbour-list totals), and out[n] receives the total.
constexpr int SS_THREADS = 1024;
constexpr int SS_MAX = SS_THREADS * 32;

__device__ __forceinline__ void scan_small_at(const uint32_t *in, uint32_t *rev,
                                              uint32_t *out, int n,
                                              uint32_t *total_dev,
                                              int write_total_at_n) {
    __shared__ uint32_t ws[SS_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int chunk = (n + SS_THREADS - 1) / SS_THREADS;   // <= 32
    const int b = threadIdx.x * chunk;
    uint32_t v[32];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int i = b + k;
        v[k] = (k < chunk && i < n) ? in[i] + (rev ? rev[i] : 0u) : 0u;
        sum += v[k];
    }
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    uint32_t pre = (w > 0 ? ws[w - 1] : 0u) + x - sum;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int i = b + k;
        if (k < chunk && i < n) {
            if (rev) rev[i] = 0;
            out[i] = pre;
            pre += v[k];
        }
    }
    if (threadIdx.x == SS_THREADS - 1) {
        if (total_dev) *total_dev = ws[SS_THREADS / 32 - 1];
        if (write_total_at_n) out[n] = ws[SS_THREADS / 32 - 1];
    }
}

__global__ void __launch_bounds__(SS_THREADS)
    k_scan_small(const uint32_t *in, uint32_t *rev, uint32_t *out, int n,
                 uint32_t *total_dev, int write_total_at_n) {
    scan_small_at(in, rev, out, n, total_dev, write_total_at_n);
}

void exclusive_scan(cudaStream_t s, const uint32_t *in, uint32_t *out, int n,
                    uint32_t *total_dev, SortScratch &sc, int *launches) {
    if (n <= 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
        return;
    }
    if (n <= SS_MAX) {
        k_scan_small<<<1, SS_THREADS, 0, s>>>(in, nullptr, out, n, total_dev, 0);
        *launches += 1;
        return;
    }
    scan_rec(s, in, out, n, total_dev, sc.scan_tmp, launches);
}

bool list_offsets_small(cudaStream_t s, const uint32_t *own, uint32_t *rev,
                        uint32_t *off, int n, int *launches) {
    if (n <= 0 || n > SS_MAX) return false;
    k_scan_small<<<1, SS_THREADS, 0, s>>>(own, rev, off, n, nullptr, 1);
    *launches += 1;
    return true;
}

// ---------------------------------------------------------------- gather --
__global__ void k_gather(int n, const uint32_t *__restrict__ perm, GatherList g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t src = perm[i];
    if (!SPH_DCHECK(src < (uint32_t)n)) return;
    for (int k = 0; k < g.nd; ++k) g.dst[k][i] = g.src[k][src];
    for (int k = 0; k < g.ni; ++k) g.idst[k][i] = g.isrc[k][src];
}

void gather_by_perm(cudaStream_t s, int n, const uint32_t *perm,
                    const GatherList &g, int *launches) {
    if (n <= 0) return;
    int bs = 256;
    k_gather<<<(n + bs - 1) / bs, bs, 0, s>>>(n, perm, g);
    *launches += 1;
}

// ------------------------------------------------------------ cell table --
__global__ void k_table_insert(int n, const uint64_t *__restrict__ skey,
                               uint64_t *tkey, uint32_t *tstart,
                               uint32_t tmask) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = skey[i];
    if (i > 0 && skey[i - 1] == k) return;
    uint32_t slot = hash_slot(k, tmask);
    // The table holds at most n keys in 2n slots, so a free slot exists and
    // the probe ends within tmask + 1 steps.
    for (uint32_t it = 0; it <= tmask; ++it) {
        unsigned long long prev = atomicCAS((unsigned long long *)&tkey[slot],
                                            (unsigned long long)EMPTY_KEY,
                                            (unsigned long long)k);
        if (prev == EMPTY_KEY || prev == k) {
            tstart[slot] = (uint32_t)i;
            return;
        }
        slot = (slot + 1) & tmask;
    }
}

__global__ void k_table_end(int n, const uint64_t *__restrict__ skey,
                            const uint64_t *__restrict__ tkey, uint32_t *tend,
                            uint32_t tmask, const double *h, float *tmaxh) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    table_mark_end(i, n, skey, tkey, tend, tmask, h, tmaxh);
}

// Gather in sorted order fused with the insertion of each cell's start.
__device__ __forceinline__ void gather_insert_at(int i, int n, const uint32_t *__restrict__ perm,
                                                 const GatherList &g,
                                                 const uint64_t *__restrict__ skey,
                                                 uint64_t *tkey, uint32_t *tstart,
                                                 uint32_t tmask) {
    if (i >= n) return;
    uint32_t src = perm[i];
    if (!SPH_DCHECK(src < (uint32_t)n)) return;
    for (int k = 0; k < g.nd; ++k) g.dst[k][i] = g.src[k][src];
    for (int k = 0; k < g.ni; ++k) g.idst[k][i] = g.isrc[k][src];
    uint64_t k = skey[i];
    if (i > 0 && skey[i - 1] == k) return;
    uint32_t slot = hash_slot(k, tmask);
    for (uint32_t it = 0; it <= tmask; ++it) {
        unsigned long long prev = atomicCAS((unsigned long long *)&tkey[slot],
                                            (unsigned long long)EMPTY_KEY,
                                            (unsigned long long)k);
        if (prev == EMPTY_KEY || prev == k) {
            tstart[slot] = (uint32_t)i;
            return;
        }
        slot = (slot + 1) & tmask;
    }
}

__global__ void k_gather_insert(int n, const uint32_t *__restrict__ perm,
                                GatherList g, const uint64_t *__restrict__ skey,
                                uint64_t *tkey, uint32_t *tstart,
                                uint32_t tmask) {
    gather_insert_at(blockIdx.x * blockDim.x + threadIdx.x, n, perm, g, skey, tkey,
                     tstart, tmask);
}

void gather_insert(cudaStream_t s, int n, const uint32_t *perm,
                   const GatherList &g, const uint64_t *skey, uint64_t *tkey,
                   uint32_t *tstart, uint32_t tmask, int *launches) {
    if (n <= 0) return;
    k_gather_insert<<<(n + 255) / 256, 256, 0, s>>>(n, perm, g, skey, tkey,
                                                     tstart, tmask);
    *launches += 1;
}

// Reset before a rebuild: level bounding boxes and mask, every table key,
// and up to four counters.
__device__ __forceinline__ void rebuild_reset_at(const RebuildReset &r, uint32_t vb,
                                                 uint32_t nvb) {
    const uint32_t t0 = vb * blockDim.x + threadIdx.x;
    const uint32_t st = nvb * blockDim.x;
    if (t0 < MAX_LEVELS * 4) r.bbox[t0] = (t0 & 1) ? -1 : 0x7fffffff;
    if (t0 == 0) *r.level_mask = 0;
    if (t0 < 5 && r.zero[t0]) *r.zero[t0] = 0;
    for (uint32_t k = t0; k < r.tslots; k += st) r.tkey[k] = EMPTY_KEY;
}

__global__ void k_rebuild_reset(RebuildReset r) { rebuild_reset_at(r, blockIdx.x, gridDim.x); }

__global__ void k_occupancy(int n, const uint64_t *__restrict__ key,
                            int lshift, const int *__restrict__ bbox,
                            uint32_t *occ) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = key[i];
    const int l = (int)(k >> lshift);
    const uint64_t m = k & ((1ull << lshift) - 1ull);
    const int ix = (int)compact2(m), iy = (int)compact2(m >> 1);
    const int *bb = bbox + 4 * l;
    const int bx = occ_block(ix, bb[0], bb[1]), by = occ_block(iy, bb[2], bb[3]);
    atomicOr(&occ[(l * OCC_N + by) * (OCC_N / 32) + (bx >> 5)], 1u << (bx & 31));
}

void launch_occupancy(cudaStream_t s, int n, const uint64_t *key, int lshift,
                      const int *bbox, uint32_t *occ, int *launches) {
    cudaMemsetAsync(occ, 0, sizeof(uint32_t) * OCC_WORDS, s);
    if (n <= 0) return;
    k_occupancy<<<(n + 255) / 256, 256, 0, s>>>(n, key, lshift, bbox, occ);
    *launches += 1;
}

// Smallest value of v over each cell of a sorted set, stored at the cell's
// first particle (other entries are left as they are).
__global__ void k_cell_min(int n, const uint64_t *__restrict__ skey,
                           const double *__restrict__ v, double *cmin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = skey[i];
    if (i > 0 && skey[i - 1] == k) return;
    double m = v[i];
    for (int j = i + 1; j < n && skey[j] == k; ++j) m = fmin(m, v[j]);
    cmin[i] = m;
}

void launch_cell_min(cudaStream_t s, int n, const uint64_t *skey,
                     const double *v, double *cmin, int *launches) {
    if (n <= 0) return;
    k_cell_min<<<(n + 255) / 256, 256, 0, s>>>(n, skey, v, cmin);
    *launches += 1;
}

int rebuild_reset_blocks(uint32_t tslots) {
    int nb = (int)std::min<uint32_t>((tslots + 255) / 256, 608u);
    return nb < 1 ? 1 : nb;
}
void launch_rebuild_reset(cudaStream_t s, const RebuildReset &r, int *launches) {
    k_rebuild_reset<<<rebuild_reset_blocks(r.tslots), 256, 0, s>>>(r);
    *launches += 1;
}

// ---------------------------------------------- batched small builds ----
// The same bodies over the work items of several instances (each item one
// block of the instance's single-launch grid); a block syncs before its
// next item, whose shared memory it reuses.
template <class Rec, class F>
__device__ __forceinline__ void batch_blocks(const Rec *args, const BatchSpan &sp, F &&f) {
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        f(args[b.q], b.vb, b.nvb);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
    k_rebuild_reset_batch(const RebuildReset *args, BatchSpan sp) {
    batch_blocks(args, sp, [](const RebuildReset &r, int vb, int nvb) {
        rebuild_reset_at(r, vb, nvb);
    });
}
__global__ void __launch_bounds__(256) k_keys_batch(const KeysRec *args, BatchSpan sp) {
    batch_blocks(args, sp, [](const KeysRec &r, int vb, int) { keys_at(r, vb); });
}
__global__ void __launch_bounds__(RSS_THREADS)
    k_radix_small_batch(const RadixSmallRec *args, BatchSpan sp) {
    batch_blocks(args, sp, [](const RadixSmallRec &r, int, int) {
        radix_small_at(r.n, r.passes, r.ka, r.va, r.kb, r.vb);
    });
}
__global__ void __launch_bounds__(256)
    k_gather_insert_batch(const GatherInsertRec *args, BatchSpan sp) {
    batch_blocks(args, sp, [](const GatherInsertRec &r, int vb, int) {
        gather_insert_at(vb * blockDim.x + threadIdx.x, r.n, r.perm, r.g, r.skey, r.tkey,
                         r.tstart, r.tmask);
    });
}
__global__ void __launch_bounds__(SS_THREADS)
    k_scan_small_batch(const ScanSmallRec *args, BatchSpan sp) {
    batch_blocks(args, sp, [](const ScanSmallRec &r, int, int) {
        scan_small_at(r.in, r.rev, r.out, r.n, r.total_dev, r.write_total_at_n);
    });
}

int radix_small_max() { return RSS_MAX; }
bool radix_small_available() { return radix_small_ready(); }
int scan_small_max() { return SS_MAX; }

template <class K>
static int resident(K kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}
static int batch_grid(int per_sm, int total) {
    const long long g = (long long)per_sm * gpu_sms();
    return (int)(g < total ? g : total);
}
void launch_rebuild_reset_batch(cudaStream_t s, const RebuildReset *args, const BatchSpan &sp) {
    static const int r = resident(k_rebuild_reset_batch, 256, 0);
    if (sp.total > 0) k_rebuild_reset_batch<<<batch_grid(r, sp.total), 256, 0, s>>>(args, sp);
}
void launch_keys_batch(cudaStream_t s, const KeysRec *args, const BatchSpan &sp) {
    static const int r = resident(k_keys_batch, 256, 0);
    if (sp.total > 0) k_keys_batch<<<batch_grid(r, sp.total), 256, 0, s>>>(args, sp);
}
bool launch_radix_small_batch(cudaStream_t s, const RadixSmallRec *args, const BatchSpan &sp,
                              int max_n) {
    static const bool ok = cudaFuncSetAttribute(k_radix_small_batch,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                RSS_MAX * 12) == cudaSuccess;
    if (!ok || max_n > RSS_MAX) {
        cudaGetLastError();
        return false;
    }
    if (sp.total > 0)
        k_radix_small_batch<<<std::min(sp.total, gpu_sms()), RSS_THREADS, (size_t)max_n * 12, s>>>(
            args, sp);
    return true;
}
void launch_gather_insert_batch(cudaStream_t s, const GatherInsertRec *args, const BatchSpan &sp) {
    static const int r = resident(k_gather_insert_batch, 256, 0);
    if (sp.total > 0) k_gather_insert_batch<<<batch_grid(r, sp.total), 256, 0, s>>>(args, sp);
}
void launch_scan_small_batch(cudaStream_t s, const ScanSmallRec *args, const BatchSpan &sp) {
    static const int r = resident(k_scan_small_batch, SS_THREADS, 0);
    if (sp.total > 0) k_scan_small_batch<<<batch_grid(r, sp.total), SS_THREADS, 0, s>>>(args, sp);
}


void build_cell_table(cudaStream_t s, int n, const uint64_t *skey,
                      uint64_t *tkey, uint32_t *tstart, uint32_t *tend,
                      uint32_t tmask, int *launches, const double *h,
                      float *tmaxh) {
    cudaMemsetAsync(tkey, 0xff, sizeof(uint64_t) * ((size_t)tmask + 1), s);
    if (n <= 0) return;
    int bs = 256;
    k_table_insert<<<(n + bs - 1) / bs, bs, 0, s>>>(n, skey, tkey, tstart, tmask);
    k_table_end<<<(n + bs - 1) / bs, bs, 0, s>>>(n, skey, tkey, tend, tmask, h,
                                                 tmaxh);
    *launches += 2;
}

SPH_DEBUG_COUNTER(debug_failures_keys_sort)

}  // namespace sph
