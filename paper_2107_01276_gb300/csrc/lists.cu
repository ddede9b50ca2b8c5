// Per-rebuild packing (levels, FP32 anchor coordinates, float mirrors) and
// the CSR neighbour lists N(i) (definition and search in neighbors.cuh).
//
// List build: one walk per particle stages its own entries and counts the
// reverse ones -> exclusive scan -> place (own entries copied, reverse
// entries written into the coarser neighbours' lists) -> sort the reverse
// segment of each list, so lists are deterministic: own entries in
// traversal order, then the finer-level entries in ascending index.
#include "debug_checks.cuh"
#include "lists.cuh"
#include "neighbors.cuh"
#include "team.cuh"

#include <algorithm>
#include <type_traits>

namespace sph {

// ------------------------------------------------------------------ pack --
__device__ __forceinline__ void pack_at(const PackArgs &a, int i) {
    a.lev[i] = (uint8_t)(a.skey[i] >> a.lshift);
    a.pk[i] = anchor_record(a.x[i], a.y[i], a.h[i], a.lo, a.Ad, a.invAd, a.an);
    if (a.tend) table_mark_end(i, a.n, a.skey, a.tkey, a.tend, a.tmask, a.h, a.tmaxh);
    if (!a.mixed) return;
    a.mf[i] = (float)a.m[i];
    a.pf[i] = (float)a.p[i];
    a.uf[i] = (float)a.u[i];
    a.vf[i] = (float)a.v[i];
}

__global__ void k_pack(PackArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    pack_at(a, i);
}

// The same over the work items of several instances (batched step).
__global__ void __launch_bounds__(BATCH_THREADS)
    k_pack_batch(const PackArgs *__restrict__ args, BatchSpan sp) {
    for (int item = blockIdx.x; item < sp.total; item += gridDim.x) {
        const int q = sp.find(item);
        const PackArgs a = args[q];
        const int i = (item - __ldg(&sp.first[q])) * BATCH_THREADS + (int)threadIdx.x;
        if (i < a.n) pack_at(a, i);
    }
}

// Anchor coordinates of a particle set (static sets: walls, background).
__global__ void k_anchor_pack(int n, const double *x, const double *y,
                              const double *h, double lo0, double lo1,
                              double A0, double A1, Anchor an, float4 *pk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lo[2] = {lo0, lo1}, A[2] = {A0, A1}, iA[2] = {1.0 / A0, 1.0 / A1};
    pk[i] = anchor_record(x[i], y[i], h[i], lo, A, iA, an);
}

// ------------------------------------------------------------ list build --
// A staged entry carries this bit when its particle lies on a coarser level
// than the row's owner (the pair also needs a reverse entry).  Particle
// indices stay below 2^31: a context holds far fewer particles.
constexpr uint32_t STAGE_COARSE = 0x80000000u;

// Membership of candidate j for particle i: FP32 anchor filter with the
// FP64 predicate in its band (exact, for both precisions).
__device__ __forceinline__ bool member(const ListArgs &a, const float4 &pi,
                                       double xi, double yi, double hi,
                                       int j) {
    float dx, dy, r2;
    if (a.skin > 1.0f) {
        // skin lists: a superset is all that is needed, and the skin is far
        // wider than the FP32 error of the separation
        const float4 pj = __ldg(&a.pk[j]);
        anchor_sep(a.an, pi, pj, dx, dy);
        const float R = a.skin * 3.0f * fmaxf(pi.z, pj.z);
        return fmaf(dx, dx, dy * dy) < R * R;
    }
    return pred_mixed(a.d, a.an, pi, __ldg(&a.pk[j]), xi, yi, hi, a.x, a.y,
                      a.h, j, dx, dy, r2);
}

// Single-walk list build: a team of T lanes walks particle i's own and
// coarser levels (per level, up to T cells looked up at once, then the
// candidates of all of them taken T at a time, one per lane); the team's
// ballot orders each group, so own entries come in (cell, index) order
// whatever T is.  They go into
// a fixed-stride staging row of stage_w entries; particles with more own
// entries go to a queue that k_list_fill_queue handles with a second walk.

template <int T>
__device__ __forceinline__ void list_gather_at(const ListArgs &a, int i, const Team<T> &tm) {
    const int li = a.lev[i];
    const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
    const float4 pi = a.pk[i];
    const float2 q = anchor_rel(a.an, pi);
    uint32_t k = 0;
    const uint32_t W = a.stage_w;
    uint32_t *row = a.stage + (size_t)i * W;
    const unsigned below = tm.mask & ((1u << (threadIdx.x & 31)) - 1u);
    for_each_candidate_team<T, true>(a.g, a.d, li, q.x, q.y, pi.z, a.skin,
                                     tm.lane, tm.mask,
                                     [](uint32_t, uint32_t) { return true; },
                                     [&](uint32_t j, bool valid) {
        const bool in = valid && member(a, pi, xi, yi, hi, (int)j);
        const unsigned bal = T == 1 ? (in ? 1u : 0u)
                                    : __ballot_sync(tm.mask, in);
        if (in) {
            const uint32_t pos = k + (T == 1 ? 0u : __popc(bal & below));
            const bool co = __ldg(&a.lev[j]) > li;
            if (pos < W) row[pos] = co ? (j | STAGE_COARSE) : j;
            if (co) atomicAdd(&a.rev[j], 1u);
        }
        k += __popc(bal);
    });
    if (tm.lane == 0) {
        a.own[i] = k;
        atomicMax(a.max_own, k);
        if (k > W) a.queue[atomicAdd(a.nqueue, 1u)] = (uint32_t)i;
    }
}

template <int T>
__global__ void __launch_bounds__(128) k_list_gather(ListArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    list_gather_at<T>(a, i, tm);
}

// Copies the staged own entries into place and writes the reverse entries
// (i into the list of each coarser neighbour j); T lanes per particle.
template <int T>
__device__ __forceinline__ void list_place_at(const ListArgs &a, int i, const Team<T> &tm) {
    const uint32_t own = a.own[i];
    if (own <= a.stage_w) {               // else handled by k_list_fill_queue
        const uint32_t base = a.off[i];
        const uint32_t *row = a.stage + (size_t)i * a.stage_w;
        const uint32_t cap = a.cap;
#pragma unroll 4
        for (uint32_t k = tm.lane; k < own; k += T) {
            const uint32_t ent = row[k];
            const uint32_t j = ent & ~STAGE_COARSE;
            if (!SPH_DCHECK(j < (uint32_t)a.n)) continue;
            if (base + k < cap) a.list[base + k] = j;
            if (ent & STAGE_COARSE) {
                const uint32_t rp = a.off[j] + a.own[j] + atomicAdd(&a.rev[j], 1u);
                if (rp < cap) a.list[rp] = (uint32_t)i;
            }
        }
    }
    if (i == a.n - 1 && tm.lane == 0 && a.off[a.n] > a.cap) atomicOr(a.overflow, 1);
}

template <int T>
__global__ void __launch_bounds__(128) k_list_place(ListArgs a) {
    const Team<T> tm;
    const int i = Team<T>::particle();
    if (i >= a.n) return;
    list_place_at<T>(a, i, tm);
}

__global__ void k_list_total(int n, const uint32_t *own, const uint32_t *rev,
                             uint32_t *tot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tot[i] = own[i] + rev[i];
}

// Second walk for the queued particles (more than stage_w own entries):
// same order as k_list_gather; teams take queue entries in turn.
template <int T>
__device__ __forceinline__ void list_fill_queue_at(const ListArgs &a, uint32_t vb,
                                                   uint32_t nvb, const Team<T> &tm) {
    const uint32_t nq = *a.nqueue;
    const uint32_t team = (vb * blockDim.x + threadIdx.x) / T;
    const uint32_t nteam = (nvb * blockDim.x) / T;
    const unsigned below = tm.mask & ((1u << (threadIdx.x & 31)) - 1u);
    for (uint32_t qi = team; qi < nq; qi += nteam) {
        const int i = (int)a.queue[qi];
        const int li = a.lev[i];
        const double xi = a.x[i], yi = a.y[i], hi = a.h[i];
        const float4 pi = a.pk[i];
        const float2 q = anchor_rel(a.an, pi);
        uint32_t k = a.off[i];
        const uint32_t cap = a.cap;
        for_each_candidate_team<T, true>(a.g, a.d, li, q.x, q.y, pi.z, a.skin,
                                         tm.lane, tm.mask,
                                         [](uint32_t, uint32_t) { return true; },
                                         [&](uint32_t j, bool valid) {
            const bool in = valid && member(a, pi, xi, yi, hi, (int)j);
            const unsigned bal = __ballot_sync(tm.mask, in);
            if (in) {
                const uint32_t pos = k + __popc(bal & below);
                if (pos < cap) a.list[pos] = j;
                if (__ldg(&a.lev[j]) > li) {
                    uint32_t rp = a.off[j] + a.own[j] + atomicAdd(&a.rev[j], 1u);
                    if (rp < cap) a.list[rp] = (uint32_t)i;
                }
            }
            k += __popc(bal);
        });
    }
}

template <int T>
__global__ void __launch_bounds__(128) k_list_fill_queue(ListArgs a) {
    const Team<T> tm;
    list_fill_queue_at<T>(a, blockIdx.x, gridDim.x, tm);
}

// ------------------------------------------------------ tiled list build --
// Cell-tiled walk: one warp takes the particles of one cell (up to 32 at a
// time, lane = particle).  For each level at or above the cell's, the warp
// looks up the cells around the bounding box of its particles once (a lane
// per cell), stages their candidates in shared memory (a batch of loads
// with no dependence between them) and every lane tests its particle
// against each staged candidate: a broadcast shared-memory read and a few
// FP32 operations per pair, instead of a lookup and a global load per
// particle.  Own entries come in (level, row, column, index) order.
//
// Separations: candidates and particles carry FP32 coordinates relative to
// the cell's first particle (anchor separations), so the pair separation is
// one subtraction.  Its error bound grows with the distance G from that
// reference; the exact-mode band below includes it.  Images on a periodic
// axis: a member j of a particle i in the cell lies within skin * c_l' +
// w_l of the reference, so while that stays below half the period the
// reference-relative image is the minimum image; otherwise (coarse levels
// of small periodic boxes) each pair is wrapped explicitly.
constexpr int TILE_CAP = 256;   // staged candidates per warp and batch
constexpr int TILE_LD = 2;      // candidate loads in flight per lane

// Squared gap between the box [xc - hx, xc + hx] x [yc - hy, yc + hy] and
// cell (cx, cy) of level L (unwrapped indices), less a margin far above
// FP32 rounding; periodic axes use the nearest image of the cell, the edge
// cells of a non-periodic axis reach to infinity.
__device__ __forceinline__ float box_gap2(const Domain &d, const Level &L,
                                          int cx, int cy, float xc, float yc,
                                          float hx, float hy) {
    const int c[2] = {cx, cy};
    const float q[2] = {xc, yc}, hh[2] = {hx, hy};
    float g2 = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const float w = L.wf[ax];
        const float m = 1e-5f * (fabsf(q[ax]) + hh[ax] + w);
        float gap;
        if (d.periodic[ax]) {
            const float P = (float)L.n[ax] * w;
            float t = q[ax] - ((float)c[ax] + 0.5f) * w;
            t -= P * rintf(t * L.invP[ax]);
            gap = fabsf(t) - 0.5f * w - hh[ax];
        } else {
            float lo = (float)c[ax] * w, hi = lo + w;
            if (c[ax] <= 0) lo = -3.0e38f;
            if (c[ax] >= L.n[ax] - 1) hi = 3.0e38f;
            gap = fmaxf(lo - (q[ax] + hh[ax]), (q[ax] - hh[ax]) - hi);
        }
        gap = fmaxf(0.0f, gap - m);
        g2 += gap * gap;
    }
    return g2;
}

// One chunk of a cell: particles p0 .. min(p0 + 32, ce) - 1 of the cell
// starting at cs (level lc); `only` >= 0 restricts the work to that one
// particle.  DIRECT = false: own entries into the staging rows, reverse
// entries counted; DIRECT = true (particles whose rows overflowed): own
// entries straight into the list at off[i], reverse entries placed.  Both
// modes take identical membership decisions (same reference, same
// per-level constants, same arithmetic); the cells a chunk visits depend
// on its bounding box, but a cell only one of them visits holds no member
// (its gap exceeds the pair radius by the pruning margin).
// sc: the warp's staging buffer (TILE_CAP entries); pcs: 20 ints of the
// warp's shared memory for the query's cell pieces.
// span: 2 when the chunk's particles lie in up to 2 x 2 neighbouring cells
// of level lc (merged chunks), else 1; the distance bound G of the FP32
// error analysis grows with it.  A particle queued for the direct pass
// records its chunk's reference and span, so that pass takes the same
// decisions with the same arithmetic.
template <bool DIRECT, int T>
__device__ __forceinline__ void tile_chunk(const ListArgs &a, float4 *sc,
                                           int *pcs, int lc, uint32_t cs,
                                           uint32_t pe, uint32_t p0, int only,
                                           int span = 1) {
    static_assert(T == 1 || T == 4 || T == 16, "team of 1, 4 or 16 lanes");
    const int lane = threadIdx.x & 31;
    const int sub = lane & (T - 1);           // lane within the particle's team
    const uint32_t i = p0 + (uint32_t)(lane / T);
    const bool act = i < pe && (only < 0 || (int)i == only);
    const float4 pC = __ldg(&a.pk[cs]);
    float rxi = 0.0f, ryi = 0.0f, Ri = 0.0f;
    float xlo = 3.0e38f, xhi = -3.0e38f, ylo = 3.0e38f, yhi = -3.0e38f, hmx = 0.0f;
    // the chunk's bounding box in reference-relative coordinates
    float rxlo = 3.0e38f, rxhi = -3.0e38f, rylo = 3.0e38f, ryhi = -3.0e38f;
    if (act) {
        const float4 pi = __ldg(&a.pk[i]);
        anchor_sep(a.an, pi, pC, rxi, ryi);
        Ri = a.skin * (3.0f * pi.z);
        const float2 q = anchor_rel(a.an, pi);
        xlo = xhi = q.x;
        ylo = yhi = q.y;
        hmx = pi.z;
        rxlo = rxhi = rxi;
        rylo = ryhi = ryi;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        xlo = fminf(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
        xhi = fmaxf(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
        ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
        yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
        hmx = fmaxf(hmx, __shfl_xor_sync(0xffffffffu, hmx, o));
        rxlo = fminf(rxlo, __shfl_xor_sync(0xffffffffu, rxlo, o));
        rxhi = fmaxf(rxhi, __shfl_xor_sync(0xffffffffu, rxhi, o));
        rylo = fminf(rylo, __shfl_xor_sync(0xffffffffu, rylo, o));
        ryhi = fmaxf(ryhi, __shfl_xor_sync(0xffffffffu, ryhi, o));
    }
    const float xc = 0.5f * (xlo + xhi), yc = 0.5f * (ylo + yhi);
    const float bx = 0.5f * (xhi - xlo), by = 0.5f * (yhi - ylo);
    const float Rmx = a.skin * (3.0f * hmx);   // largest pair radius of a chunk particle
    const uint32_t W = a.stage_w;
    uint32_t k = 0;
    if (DIRECT && act) k = a.off[i];
    uint32_t *row = a.stage + (size_t)i * W;
    const Level &LC = a.g.lev[lc];
    const float Amax = fmaxf(a.an.A[0], a.an.A[1]);
    const float Lx = (float)a.d.L[0], Ly = (float)a.d.L[1];
    const float iLx = 1.0f / Lx, iLy = 1.0f / Ly;
    const bool exact = !(a.skin > 1.0f);
    const uint32_t lmask = a.g.level_mask & ~((1u << lc) - 1u);
    for (uint32_t mm = lmask; mm; mm &= mm - 1) {
        const int l = __ffs(mm) - 1;
        const int *bb = a.g.bbox + 4 * l;
        if (__ldg(&bb[0]) > __ldg(&bb[1])) continue;   // level holds no particle
        const Level &L = a.g.lev[l];
        const float Rl = a.skin * fmaxf(3.0f * hmx, L.cf);
        const float Q = Rl * (1.0f + 1e-5f);
        AxisPieces px, py;
        if (!axis_pieces(a.d, L, bb, 0, xc, bx + Q, px)) continue;
        if (!axis_pieces(a.d, L, bb, 1, yc, by + Q, py)) continue;
        // per-level constants (functions of lc and l only)
        const float reach = a.skin * L.cf + (float)span * fmaxf(LC.wf[0], LC.wf[1]) +
                            fmaxf(L.wf[0], L.wf[1]);
        const bool wrapx = a.d.periodic[0] && 2.0f * (reach + 4.0f * a.an.A[0]) >= Lx;
        const bool wrapy = a.d.periodic[1] && 2.0f * (reach + 4.0f * a.an.A[1]) >= Ly;
        const bool wrap = wrapx || wrapy;
        const float G = reach + (wrap ? fmaxf(Lx, Ly) : 0.0f);
        const float KB = 4.0f * Amax + G;
        const bool coarse = l > lc;
        // the query's cell pieces go to shared memory: nothing of them stays
        // in registers through the staging and test loops
        __syncwarp();
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                pcs[t] = px.first[t];
                pcs[3 + t] = px.shift[t];
                pcs[6 + t] = max(0, px.last[t] - px.first[t] + 1);
                pcs[9 + t] = py.first[t];
                pcs[12 + t] = py.shift[t];
                pcs[15 + t] = max(0, py.last[t] - py.first[t] + 1);
            }
        }
        __syncwarp();
        const int nx = pcs[6] + pcs[7] + pcs[8];
        const int ncell = nx * (pcs[15] + pcs[16] + pcs[17]);
        const uint64_t lbits = (uint64_t)l << (2 * a.g.mbits);
        for (int base = 0; base < ncell; base += 32) {
            // lane -> one cell of the query (row-major, unwrapped order)
            uint32_t s = 0, e = 0;
            const int idx = base + lane;
            if (idx < ncell) {
                const int iy = idx / nx;
                int ix = idx - iy * nx, jy = iy;
                int kx = 0, ky = 0;
                while (kx < 2 && ix >= pcs[6 + kx]) ix -= pcs[6 + kx++];
                while (ky < 2 && jy >= pcs[15 + ky]) jy -= pcs[15 + ky++];
                const int cx = pcs[kx] + ix, sx = pcs[3 + kx];
                const int cy = pcs[9 + ky] + jy, sy = pcs[12 + ky];
                const float g2 = box_gap2(a.d, L, cx, cy, xc, yc, bx, by);
                float hc;
                if (g2 < Rl * Rl &&
                    table_lookup(a.g, lbits | (spread2((uint64_t)(cy + sy)) << 1) |
                                          spread2((uint64_t)(cx + sx)),
                                 s, e, &hc)) {
                    const float Rc = a.skin * 3.0f * fmaxf(hmx, hc);
                    if (!(g2 < Rc * Rc)) s = e = 0;
                    if (!SPH_DCHECK(s <= e && e <= (uint32_t)a.n)) s = e = 0;
                } else {
                    s = e = 0;
                }
            }
            const uint32_t cnt = e - s;
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
            const uint32_t exc = inc - cnt;
            for (uint32_t q0 = 0; q0 < total; q0 += TILE_CAP) {
                const uint32_t mq = min((uint32_t)TILE_CAP, total - q0);
                // stage: candidate q0 + u; its cell is the first lane whose
                // inclusive count exceeds it (binary search over the lanes),
                // TILE_LD independent loads per lane in flight.  Candidates
                // farther from the chunk's bounding box than the largest
                // pair radius they could have (with a margin far above FP32
                // error) are no member of any particle of the chunk and are
                // not staged; the others keep their order (ballot
                // compaction), so the test loop sees the same members in the
                // same order.
                uint32_t m = 0;
                for (uint32_t u0 = 0; u0 < mq; u0 += 32 * TILE_LD) {
                    float4 v[TILE_LD];
                    uint32_t jj[TILE_LD];
#pragma unroll
                    for (int r = 0; r < TILE_LD; ++r) {
                        const uint32_t u = u0 + 32 * r + lane;
                        const uint32_t qq = q0 + min(u, mq - 1);
                        int pos = 0;
#pragma unroll
                        for (int st = 16; st; st >>= 1) {
                            const uint32_t vv = __shfl_sync(0xffffffffu, inc, pos + st - 1);
                            if (vv <= qq) pos += st;
                        }
                        const uint32_t st0 = __shfl_sync(0xffffffffu, s, pos);
                        const uint32_t ex0 = __shfl_sync(0xffffffffu, exc, pos);
                        jj[r] = st0 + (qq - ex0);
                        if (u < mq) v[r] = __ldg(&a.pk[jj[r]]);
                    }
#pragma unroll
                    for (int r = 0; r < TILE_LD; ++r) {
                        const uint32_t u = u0 + 32 * r + lane;
                        float rx = 0.0f, ry = 0.0f, Rj = 0.0f;
                        bool keep = false;
                        if (u < mq) {
                            anchor_sep(a.an, v[r], pC, rx, ry);
                            Rj = a.skin * (3.0f * v[r].z);
                            keep = true;
                            if (!wrap) {
                                const float gx = fmaxf(fmaxf(rxlo - rx, rx - rxhi), 0.0f);
                                const float gy = fmaxf(fmaxf(rylo - ry, ry - ryhi), 0.0f);
                                const float Rm = fmaxf(Rmx, Rj) * 1.01f;
                                keep = fmaf(gx, gx, gy * gy) < Rm * Rm;
                            }
                        }
                        const unsigned kb = __ballot_sync(0xffffffffu, keep);
                        if (keep)
                            sc[m + (uint32_t)__popc(kb & ((1u << lane) - 1u))] =
                                make_float4(rx, ry, Rj, __uint_as_float(jj[r]));
                        m += (uint32_t)__popc(kb);
                    }
                }
                __syncwarp();
                {
                    // one loop per (exact, wrap, coarse) case, branch-free in
                    // the common ones: a predicated store and a counter.  A
                    // team of T lanes takes T consecutive candidates per
                    // iteration; the ballot keeps the team's entries in
                    // candidate order.
                    auto test = [&](auto ex_c, auto wr_c, auto co_c) {
                        constexpr bool EX = decltype(ex_c)::value;
                        constexpr bool WR = decltype(wr_c)::value;
                        constexpr bool CO = decltype(co_c)::value;
                        auto pair_in = [&](uint32_t u, uint32_t &j) {
                            const float4 c = sc[u];
                            float dx = rxi - c.x, dy = ryi - c.y;
                            if (WR) {
                                if (wrapx) dx -= Lx * rintf(dx * iLx);
                                if (wrapy) dy -= Ly * rintf(dy * iLy);
                            }
                            const float r2 = fmaf(dx, dx, dy * dy);
                            const float R = fmaxf(Ri, c.z);
                            const float R2 = R * R;
                            j = __float_as_uint(c.w);
                            bool in = r2 < R2;
                            if (EX) {
                                const float band = fmaf(R, KB, R2) * (1.0f / 65536.0f);
                                in = r2 < R2 - band;
                                if (!in && !(r2 > R2 + band))
                                    in = pred_fp64(a.d, __ldg(&a.x[i]), __ldg(&a.y[i]),
                                                   __ldg(&a.h[i]), __ldg(&a.x[j]),
                                                   __ldg(&a.y[j]), __ldg(&a.h[j]));
                            }
                            return in;
                        };
                        auto put = [&](uint32_t pos, uint32_t j) {
                            if (DIRECT) {
                                if (pos < a.cap) a.list[pos] = j;
                                if (CO) {
                                    const uint32_t rp = a.off[j] + a.own[j] +
                                                        atomicAdd(&a.rev[j], 1u);
                                    if (rp < a.cap) a.list[rp] = i;
                                }
                            } else {
                                if (pos < W) row[pos] = CO ? (j | STAGE_COARSE) : j;
                                if (CO) atomicAdd(&a.rev[j], 1u);
                            }
                        };
                        if constexpr (T == 1) {
                            if (!act) return;
#pragma unroll 4
                            for (uint32_t u = 0; u < m; ++u) {
                                uint32_t j;
                                const bool in = pair_in(u, j);
                                if (DIRECT) {
                                    if (in) put(k, j);
                                } else {
                                    if (in && k < W) row[k] = CO ? (j | STAGE_COARSE) : j;
                                    if (CO && in) atomicAdd(&a.rev[j], 1u);
                                }
                                k += in ? 1u : 0u;
                            }
                        } else {
                            const unsigned gsh = (unsigned)(lane & ~(T - 1));
                            const unsigned below = (1u << sub) - 1u;
                            for (uint32_t u0 = 0; u0 < m; u0 += T) {
                                const uint32_t u = u0 + (uint32_t)sub;
                                uint32_t j = 0;
                                const bool in = act && u < m && pair_in(u, j);
                                const unsigned gb = (__ballot_sync(0xffffffffu, in) >> gsh) &
                                                    ((1u << T) - 1u);
                                if (in) put(k + (uint32_t)__popc(gb & below), j);
                                k += (uint32_t)__popc(gb);
                            }
                        }
                    };
                    using TT = std::true_type;
                    using FF = std::false_type;
                    if (exact) {
                        if (wrap) {
                            if (coarse) test(TT(), TT(), TT()); else test(TT(), TT(), FF());
                        } else {
                            if (coarse) test(TT(), FF(), TT()); else test(TT(), FF(), FF());
                        }
                    } else {
                        if (wrap) {
                            if (coarse) test(FF(), TT(), TT()); else test(FF(), TT(), FF());
                        } else {
                            if (coarse) test(FF(), FF(), TT()); else test(FF(), FF(), FF());
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    if (!DIRECT) {
        uint32_t km = act ? k : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
        if (act && sub == 0) {
            a.own[i] = k;
            if (k > W) {
                const uint32_t q = atomicAdd(a.nqueue, 1u);
                a.queue[q] = i;
                a.qref[q] = cs | (span > 1 ? 0x80000000u : 0u);
            }
        }
        if (lane == 0 && km > 0) atomicMax(a.max_own, km);
    }
}

// Stage-mode walk.  T = 1: warp w owns the cells whose first particle lies
// in [32 w, 32 w + 32) and takes them one after another, 32 particles at a
// time.  T > 1 (small sets, where that leaves most of the GPU idle): warp w
// takes the 32 / T particles [w P, w P + P), P = 32 / T, one piece per cell
// they fall in.
// resident 128-thread blocks per SM the merged-chunk walk is compiled for
// (80 registers; measured 23 % faster than the unbounded 94 and 4-6 %
// faster than seven or eight blocks, which spill); the cell-per-chunk
// forms keep the 72 / 80 registers they were measured at
#ifndef SPH_TILE_MERGE_BLOCKS
#define SPH_TILE_MERGE_BLOCKS 6
#endif
template <int T, bool MERGE = false>
__global__ void __launch_bounds__(128, MERGE ? SPH_TILE_MERGE_BLOCKS : (T == 1 ? 7 : 6))
    k_list_tile(ListArgs a) {
    __shared__ float4 sbuf[4][TILE_CAP];
    __shared__ int spcs[4][20];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * 4u + (uint32_t)w;
    const uint32_t n = (uint32_t)a.n;
    if constexpr (T == 1) {
        const uint32_t base = gw * 32u;
        if (base >= n) return;
        const uint32_t i = base + lane;
        const bool head = i < n && (i == 0 || a.skey[i] != a.skey[i - 1]);
        unsigned heads = __ballot_sync(0xffffffffu, head);
        const uint64_t cmask = (1ull << (2 * a.g.mbits)) - 1ull;
        while (heads) {
            const uint32_t hd = base + (uint32_t)(__ffs(heads) - 1);
            heads &= heads - 1;
            const uint64_t K = a.skey[hd];
            uint32_t cs = hd, ce = hd + 1;
            table_lookup(a.g, K, cs, ce);
            const int lc = a.lev[hd];
            int span = 1;
            if constexpr (MERGE) {
                // the following cells of this warp's range join the chunk
                // while they are of the same level, within one cell of the
                // first on both axes (no wrap) and the chunk holds at most
                // 32 particles
                const uint32_t fx = compact2(K & cmask), fy = compact2((K & cmask) >> 1);
                while (ce - cs < 32 && ce < base + 32 && ce < n) {
                    const uint64_t K2 = a.skey[ce];
                    if ((K2 >> (2 * a.g.mbits)) != (K >> (2 * a.g.mbits))) break;
                    const int dx = (int)compact2(K2 & cmask) - (int)fx;
                    const int dy = (int)compact2((K2 & cmask) >> 1) - (int)fy;
                    if (dx < -1 || dx > 1 || dy < -1 || dy > 1) break;
                    uint32_t s2 = ce, e2 = ce + 1;
                    table_lookup(a.g, K2, s2, e2);
                    if (e2 - cs > 32) break;
                    heads &= ~(1u << (ce - base));
                    ce = e2;
                    span = 2;
                }
            }
            for (uint32_t p0 = cs; p0 < ce; p0 += 32)
                tile_chunk<false, 1>(a, sbuf[w], spcs[w], lc, cs, min(ce, p0 + 32), p0, -1,
                                     span);
        }
    } else {
        constexpr uint32_t P = 32 / T;
        const uint32_t w0 = gw * P;
        if (w0 >= n) return;
        const uint32_t w1 = min(n, w0 + P);
        uint32_t t = w0;
        while (t < w1) {
            const uint64_t K = a.skey[t];
            uint32_t cs = t, ce = t + 1;
            table_lookup(a.g, K, cs, ce);
            const uint32_t pe = min(ce, w1);
            tile_chunk<false, T>(a, sbuf[w], spcs[w], a.lev[t], cs, pe, t, -1);
            t = pe;
        }
    }
}

// Direct-mode pass for the particles whose own entries overflowed their
// staging row; a warp per queued particle.
__global__ void __launch_bounds__(128) k_list_tile_queue(ListArgs a) {
    __shared__ float4 sbuf[4][TILE_CAP];
    __shared__ int spcs[4][20];
    const int w = threadIdx.x >> 5;
    const uint32_t nq = *a.nqueue;
    const uint32_t gw = blockIdx.x * 4u + (uint32_t)w, nw = gridDim.x * 4u;
    for (uint32_t q = gw; q < nq; q += nw) {
        const uint32_t i = a.queue[q];
        // the reference and span of the chunk that queued it
        const uint32_t r = a.qref[q];
        const uint32_t cs = r & 0x7fffffffu;
        tile_chunk<true, 16>(a, sbuf[w], spcs[w], a.lev[i], cs, i + 1, i, (int)i,
                             (r & 0x80000000u) ? 2 : 1);
    }
}

// Sort of each reverse segment (ascending index).  Segments of at most 32
// entries (the common case: only particles next to a finer level have
// any) are sorted in registers by the particle's thread; longer ones are
// queued for a warp-wide bitonic sort in shared memory.
constexpr int SORT_REG = 32;
constexpr int SORT_SMEM = 1024;

// Ascending sort of seg[0 .. len) (len <= K) in registers: odd-even
// transposition over K slots, fixed indices, padding at the top.
template <int K>
__device__ __forceinline__ void sort_regs(uint32_t *seg, uint32_t len) {
    uint32_t r[K];
#pragma unroll
    for (int t = 0; t < K; ++t) r[t] = t < (int)len ? seg[t] : 0xffffffffu;
#pragma unroll
    for (int round = 0; round < K; ++round) {
#pragma unroll
        for (int t = round & 1; t + 1 < K; t += 2) {
            const uint32_t lo = min(r[t], r[t + 1]), hi = max(r[t], r[t + 1]);
            r[t] = lo;
            r[t + 1] = hi;
        }
    }
#pragma unroll
    for (int t = 0; t < K; ++t)
        if (t < (int)len) seg[t] = r[t];
}

__device__ __forceinline__ void list_sort_rev_at(int i, int n, const uint32_t *off,
                                                 const uint32_t *own, uint32_t *list,
                                                 uint32_t cap, uint32_t *longq,
                                                 uint32_t *nlong) {
    if (i >= n) return;
    const uint32_t b = off[i] + (own ? own[i] : 0u), e = off[i + 1];
    if (e > cap || e <= b + 1) return;
    const uint32_t len = e - b;
    if (len > SORT_REG) {
        longq[atomicAdd(nlong, 1u)] = (uint32_t)i;
        return;
    }
    // the network no wider than the segment needs (most are short)
    if (len <= 8)
        sort_regs<8>(list + b, len);
    else if (len <= 16)
        sort_regs<16>(list + b, len);
    else
        sort_regs<SORT_REG>(list + b, len);
}

__global__ void k_list_sort_rev(int n, const uint32_t *off, const uint32_t *own,
                                uint32_t *list, uint32_t cap, uint32_t *longq,
                                uint32_t *nlong) {
    list_sort_rev_at(blockIdx.x * blockDim.x + threadIdx.x, n, off, own, list, cap, longq,
                     nlong);
}

__device__ __forceinline__ void list_sort_long_at(const uint32_t *off, const uint32_t *own,
                                                  uint32_t *list, const uint32_t *longq,
                                                  const uint32_t *nlong, uint32_t vb,
                                                  uint32_t nvb) {
    __shared__ uint32_t buf[4][SORT_SMEM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *s = buf[w];
    const uint32_t nq = *nlong;
    const uint32_t gw = vb * 4 + w, nw = nvb * 4;
    for (uint32_t q = gw; q < nq; q += nw) {
        const uint32_t i = longq[q];
        const uint32_t b = off[i] + (own ? own[i] : 0u), e = off[i + 1];
        const uint32_t len = e - b;
        if (len > SORT_SMEM) {
            // rare: plain insertion sort by one lane
            if (lane == 0) {
                for (uint32_t k = b + 1; k < e; ++k) {
                    uint32_t v = list[k], m = k;
                    while (m > b && list[m - 1] > v) {
                        list[m] = list[m - 1];
                        --m;
                    }
                    list[m] = v;
                }
            }
            __syncwarp();
            continue;
        }
        uint32_t P = 32;
        while (P < len) P <<= 1;
        for (uint32_t t = lane; t < P; t += 32) s[t] = t < len ? list[b + t] : 0xffffffffu;
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t t = lane; t < P; t += 32) {
                    uint32_t ixj = t ^ j;
                    if (ixj > t) {
                        uint32_t x0 = s[t], x1 = s[ixj];
                        bool asc = (t & k) == 0;
                        if ((x0 > x1) == asc) {
                            s[t] = x1;
                            s[ixj] = x0;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (uint32_t t = lane; t < len; t += 32) list[b + t] = s[t];
        __syncwarp();
    }
}

__global__ void k_list_sort_long(const uint32_t *off, const uint32_t *own,
                                 uint32_t *list, const uint32_t *longq,
                                 const uint32_t *nlong) {
    list_sort_long_at(off, own, list, longq, nlong, blockIdx.x, gridDim.x);
}

// ---------------------------------------------- batched small builds ----
// The single-instance bodies over the work items of several instances
// (one item: one block of the instance's single-launch grid, or of a
// smaller grid where the body's results do not depend on it).
template <int T>
__global__ void __launch_bounds__(128) k_list_gather_batch(const ListArgs *args, BatchSpan sp) {
    const Team<T> tm;
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        const ListArgs &a = args[b.q];
        const int i = b.vb * (128 / T) + (int)threadIdx.x / T;
        if (i < a.n) list_gather_at<T>(a, i, tm);
    }
}
template <int T>
__global__ void __launch_bounds__(128) k_list_place_batch(const ListArgs *args, BatchSpan sp) {
    const Team<T> tm;
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        const ListArgs &a = args[b.q];
        const int i = b.vb * (128 / T) + (int)threadIdx.x / T;
        if (i < a.n) list_place_at<T>(a, i, tm);
    }
}
__global__ void __launch_bounds__(128) k_list_fill_queue_batch(const ListArgs *args, BatchSpan sp) {
    const Team<16> tm;
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        list_fill_queue_at<16>(args[b.q], b.vb, b.nvb, tm);
    }
}
__global__ void __launch_bounds__(256) k_list_sort_rev_batch(const SortSegRec *args, BatchSpan sp) {
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        const SortSegRec &r = args[b.q];
        list_sort_rev_at(b.vb * 256 + (int)threadIdx.x, r.n, r.off, r.own, r.list, r.cap, r.longq,
                         r.nlong);
    }
}
__global__ void __launch_bounds__(128) k_list_sort_long_batch(const SortSegRec *args, BatchSpan sp) {
    for (int it = blockIdx.x; it < sp.total; it += gridDim.x) {
        const BatchItem b = batch_item(sp, it);
        const SortSegRec &r = args[b.q];
        list_sort_long_at(r.off, r.own, r.list, r.longq, r.nlong, b.vb, b.nvb);
        __syncthreads();
    }
}

// ------------------------------------------------------------- launchers --
static inline int nblk_s(int n, int bs) { return (n + bs - 1) / bs; }

void sort_segments(cudaStream_t s, int n, const uint32_t *off, uint32_t *list,
                   uint32_t cap, uint32_t *longq, uint32_t *nlong,
                   int *launches) {
    if (n <= 0) return;
    k_list_sort_rev<<<nblk_s(n, 256), 256, 0, s>>>(n, off, nullptr, list, cap,
                                                   longq, nlong);
    k_list_sort_long<<<std::max(1, std::min(152 * 16, nblk_s(n, 4))), 128, 0, s>>>(
        off, nullptr, list, longq, nlong);
    *launches += 2;
}
static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

void launch_pack_batch(cudaStream_t s, const PackArgs *args, const BatchSpan &sp,
                       int blocks) {
    if (sp.total > 0)
        k_pack_batch<<<std::min(blocks, sp.total), BATCH_THREADS, 0, s>>>(args, sp);
}
int pack_batch_blocks_per_sm() {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pack_batch, BATCH_THREADS, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm;
}
void launch_pack(cudaStream_t s, const PackArgs &a) {
    if (a.n > 0) k_pack<<<nblk(a.n, 256), 256, 0, s>>>(a);
}
void launch_anchor_pack(cudaStream_t s, int n, const double *x,
                        const double *y, const double *h, const double *lo,
                        const double *A, const Anchor &an, float4 *pk) {
    if (n > 0)
        k_anchor_pack<<<nblk(n, 256), 256, 0, s>>>(n, x, y, h, lo[0], lo[1],
                                                    A[0], A[1], an, pk);
}

// Walk choice by set size (measured on GB300 over uniform and graded
// lattices of 5k to 16M particles): below ~12k particles the per-particle
// team walk keeps more warps in flight than the cell tiles; from there the
// tiles win, with teams of 4 lanes up to 48k particles (1.5x faster than
// the merged one-lane tiles at 12k-26k on uniform vortices, even at
// 36k-50k) and merged one-lane tiles beyond (0.78x the 4-lane tiles at
// 70k, 0.5x at 290k).  A.walk overrides it (tuning).
static int walk_kind(const ListArgs &a) {
    if (a.walk >= 1 && a.walk <= 4) return a.walk;
    return a.n < 12000 ? 1 : a.n < 48000 ? 2 : 4;
}

int list_walk_kind(const ListArgs &a) { return walk_kind(a); }
int list_place_team(int n) { return std::max(team_size(n), 16); }
int fill_queue_blocks() { return 4; }
int sort_long_blocks(int n) { return std::max(1, std::min(8, nblk(n, 4))); }

template <class K>
static int batch_grid_of(K kernel, int threads, int total) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long g = (long long)per_sm * gpu_sms();
    return (int)(g < total ? g : total);
}
void launch_list_gather_batch(cudaStream_t s, int team, const ListArgs *args, const BatchSpan &sp) {
    if (sp.total <= 0) return;
    with_team_or(team, 1 << 30, [&](auto t) {
        constexpr int T = decltype(t)::value;
        static const int g = batch_grid_of(k_list_gather_batch<T>, 128, 1 << 30);
        k_list_gather_batch<T><<<std::min(g, sp.total), 128, 0, s>>>(args, sp);
    });
}
void launch_list_place_batch(cudaStream_t s, int team, const ListArgs *args, const BatchSpan &sp) {
    if (sp.total <= 0) return;
    with_team_or(team, 1 << 30, [&](auto t) {
        constexpr int T = decltype(t)::value;
        static const int g = batch_grid_of(k_list_place_batch<T>, 128, 1 << 30);
        k_list_place_batch<T><<<std::min(g, sp.total), 128, 0, s>>>(args, sp);
    });
}
void launch_list_fill_queue_batch(cudaStream_t s, const ListArgs *args, const BatchSpan &sp) {
    static const int g = batch_grid_of(k_list_fill_queue_batch, 128, 1 << 30);
    if (sp.total > 0) k_list_fill_queue_batch<<<std::min(g, sp.total), 128, 0, s>>>(args, sp);
}
void launch_list_sort_rev_batch(cudaStream_t s, const SortSegRec *args, const BatchSpan &sp) {
    static const int g = batch_grid_of(k_list_sort_rev_batch, 256, 1 << 30);
    if (sp.total > 0) k_list_sort_rev_batch<<<std::min(g, sp.total), 256, 0, s>>>(args, sp);
}
void launch_list_sort_long_batch(cudaStream_t s, const SortSegRec *args, const BatchSpan &sp) {
    static const int g = batch_grid_of(k_list_sort_long_batch, 128, 1 << 30);
    if (sp.total > 0) k_list_sort_long_batch<<<std::min(g, sp.total), 128, 0, s>>>(args, sp);
}

void launch_list_walk(cudaStream_t s, const ListArgs &a, int *launches) {
    const int n = a.n;
    if (n <= 0) return;
    const int kind = walk_kind(a);
    if (kind == 3) {
        k_list_tile<1><<<nblk(n, 128), 128, 0, s>>>(a);
    } else if (kind == 4) {
        k_list_tile<1, true><<<nblk(n, 128), 128, 0, s>>>(a);
    } else if (kind == 2) {
        k_list_tile<4><<<nblk(n, 32), 128, 0, s>>>(a);
    } else {
        with_team(n, [&](auto t) {
            constexpr int T = decltype(t)::value;
            k_list_gather<T><<<nblk(n * T, 128), 128, 0, s>>>(a);
        });
    }
    *launches += 1;
}

void list_offsets(cudaStream_t s, const ListArgs &a, SortScratch &sc,
                  uint32_t *tot_tmp, int *launches) {
    const int n = a.n;
    if (n <= 0) {
        cudaMemsetAsync(a.off, 0, sizeof(uint32_t), s);
        return;
    }
    if (list_offsets_small(s, a.own, a.rev, a.off, n, launches)) return;
    k_list_total<<<nblk(n, 256), 256, 0, s>>>(n, a.own, a.rev, tot_tmp);
    // off has n + 1 entries: scan n + 1 values with a trailing zero
    cudaMemsetAsync(tot_tmp + n, 0, sizeof(uint32_t), s);
    exclusive_scan(s, tot_tmp, a.off, n + 1, nullptr, sc, launches);
    cudaMemsetAsync(a.rev, 0, sizeof(uint32_t) * n, s);
    *launches += 1;
}

void build_lists_fill(cudaStream_t s, ListArgs a, bool mixed, bool queue,
                      int *launches) {
    (void)mixed;
    const int n = a.n;
    if (n <= 0) return;
    // at least 16 lanes per particle: a list's entries are then read from
    // the staging row and written to the list in 64-byte runs
    with_team(n, [&](auto t) {
        constexpr int T = decltype(t)::value;
        k_list_place<T><<<nblk(n * T, 128), 128, 0, s>>>(a);
    }, 16);
    if (queue) {
        if (walk_kind(a) != 1)
            k_list_tile_queue<<<152 * 4, 128, 0, s>>>(a);
        else
            k_list_fill_queue<16><<<152 * 4, 128, 0, s>>>(a);
    }
    k_list_sort_rev<<<nblk(n, 256), 256, 0, s>>>(n, a.off, a.own, a.list, a.cap,
                                                  a.longq, a.nlong);
    // up to one warp per particle (4 per block): the long segments are
    // sorted in parallel whatever their number; idle warps exit at once
    k_list_sort_long<<<std::max(1, std::min(152 * 16, nblk(n, 4))), 128, 0, s>>>(
        a.off, a.own, a.list, a.longq, a.nlong);
    *launches += 4;
}

SPH_DEBUG_COUNTER(debug_failures_lists)

}  // namespace sph
