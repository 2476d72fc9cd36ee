// Least energy progress measure on the GPU: initialisation and the
// persistent frontier fixpoint (arXiv 1710.03647, Algorithm 3 semantics with
// the lifting operator of Def. "Lifting Operator" and the bound of Sec. 3.1).
//
// One round of the fixpoint kernel has two phases separated by grid barriers:
//
//   pull: every player-0 vertex v in the pull list is lifted in place,
//         f(v) <- max(f(v), min over (v,u) of f(u) (-) w(v,u));
//         if f(v) rose, v joins this round's push list.
//   push: for every vertex v of the push list and every predecessor p with
//         edge (p, v):  t = f(v) (-) w(p, v).
//           p in V1: f(p) <- max(f(p), t) with atomicMax (p's lift is a max,
//                    and t never exceeds the least fixpoint at p, because
//                    f(v) does not exceed it at v -- the soundness argument of
//                    Sec. 4: lifts never decrease f); if f(p) rose, p joins
//                    the next push list.
//           p in V0: if f(p) < t, p may need a lift (the filter of
//                    Algorithm 1's predecessor loop); p joins the next pull
//                    list.
//         A bitmap per round parity keeps each vertex at most once per list.
//
// The kernel stops when both next lists are empty: then every player-1
// vertex satisfies f(p) >= f(v) (-) w for all successors (each rise of f(v)
// was pushed) and every player-0 vertex has a successor with
// f(p) >= f(v) (-) w (otherwise the filter enqueued it and its lift restored
// one), so f is an EPM reached from 0 by sound lifts: the least one.
//
// Lists store, per entry, the exclusive prefix of their works (edges to
// scan), written at append time by one 64-bit atomic per warp, so each phase
// splits its edges evenly across all warps (merge-path style) without a
// separate scan: a warp finds its first entry by a 32-ary search and walks
// entries in windows of 32.  A player-0 lift cut by a warp boundary merges
// its partial minima through per-vertex scratch (acc, acc_done); the warp
// that completes the count finishes the lift.
//
// The lift starts from f = 0 except at warm-start vertices, which start at
// TOP (k_seed, and the proofs of the certified trials); every start is at or
// below the least fixpoint, so the argument above still gives the least one.
//
// What the file holds, in order:
//   kernels      k_bound, k_seed (warm start), k_init, the pull and push
//                phases with per-warp local worklists, k_fixpoint
//   solve        one game (eg_solve_credit): a first attempt with a short
//                round budget, then certified trial caps (dual lifts with
//                swapped owners, capped lifts, k_mark_finite,
//                k_count_undecided) if the game needs them
//   plans        batched solves of many instances in one launch (eg_plan_*),
//                with per-instance certified trials
//   resident     the resident solve behind the server (eg_server.cu)
//   noalloc      eg_solve_credit_noalloc over a fixed device array
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

constexpr unsigned long long BARRIER_LIMIT_NS = 5000000000ull;  // 5 s per wait
constexpr int LOCAL_CAP = 256;  // entries of a warp's local worklist
#ifndef EG_FIXPOINT_MIN_BLOCKS
#define EG_FIXPOINT_MIN_BLOCKS 4  // resident blocks per SM the fixpoint kernel's registers must allow
#endif

__device__ __forceinline__ int xchg(int *p, int v) { return atomicExch(p, v); }
__device__ __forceinline__ long long xchg(long long *p, long long v) {
    return (long long)atomicExch((unsigned long long *)p, (unsigned long long)v);
}

// Instances of a batched solve: instance i owns credits [fbase[i], fbase[i+1])
// and views arena vertices v = g - delta[i] (credit index g) under the map
// w' = scale[i] * w - shift[i] with bound C[i].
struct InstTable {
    int count;
    int uniform_n;     // > 0: every instance holds uniform_n credits (instance = g / uniform_n)
    const int *fbase;  // count + 1
    const int *delta;
    const long long *scale;
    const long long *shift;
    const long long *C;
    const int *inst_id;  // non-null: instance of each credit (resident solves)
    const int *active;   // non-null: instances with active[i] == 0 are left as they are
    const int *lut = nullptr;  // non-null: instance of credit b << lut_shift, for every b; a block of
    int lut_shift = 0;         //   2^lut_shift credits is no longer than the shortest instance
};

template <typename T>
struct Args {
    DevArena A;
    WeightView W;      // the single instance's view (MULTI = false)
    InstTable I;       // the instances (MULTI = true)
    int nf;            // credits: n (single) or the sum over instances
    T *f;
    int *pull_items[2];
    int *pull_offs[2];
    int *push_items[2];
    int *push_offs[2];
    unsigned *bits_pull[2];  // dedupe of the pull list of round parity k
    unsigned *bits_push[2];  // dedupe of the push list of round parity k
    const unsigned *seed_bits;  // warm start: vertices that start at TOP (or null)
    const unsigned *frozen;     // vertices held at 0 and never lifted (or null): proven player-1
                                // vertices in a dual lift of the certified trials
    unsigned inv;      // 1: owners swapped (the dual game of a certified solve), else 0
    T *acc;
    int *acc_done;
    Ctrl *ctrl;
    long long max_rounds;  // round the kernel stops at (0: none)
    long long r0;          // first round (resident solves resume where the last slice stopped)
    int slice;             // 1: stopping at max_rounds or at the doorbell is not an error
    const volatile unsigned *doorbell;  // resident solves: host-set flag that ends the slice
    int local_windows;  // per-warp budget of local windows per round (0: no chaining)
    int local_maxdeg;   // largest degree a vertex may have to be chained locally
    int chunk;          // edges per chunk of a list with more than that per warp (0: one chunk per warp)
    unsigned long long wait_ns;  // limit of each grid-barrier wait
    const int *level;  // SCC-ordered solves: topological level of each vertex (or null)
    int cur_level;     // the level being solved; predecessors above it are left for later
    const int *tiles;  // non-null: the 32-credit tiles (index g >> 5) the O(n) passes visit, ascending
    long long ntiles;  //   and how many (the tiles covering the instances a batched lift works on)
};

// One instance's view of the arena, carried per list entry.  A negative C
// marks an instance whose solve was taken over elsewhere (a resident solve
// retires it): its entries are consumed without work.
struct View {
    int delta;
    long long scale;
    long long shift;
    long long C;
};

__device__ __forceinline__ long long wmapv(int w, const View &v) { return v.scale * (long long)w - v.shift; }

__device__ __forceinline__ int inst_of(const InstTable &I, int g) {
    if (I.inst_id) return __ldg(I.inst_id + g);
    if (I.uniform_n > 0) return g / I.uniform_n;
    if (I.lut) {  // the instance of the block's first credit, or the next one
        int i = __ldg(I.lut + (g >> I.lut_shift));
        while (__ldg(I.fbase + i + 1) <= g) ++i;
        return i;
    }
    int lo = 0, hi = I.count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(I.fbase + mid) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <bool MULTI, typename T>
__device__ __forceinline__ View view_of(const Args<T> &a, int g) {
    if (!MULTI) return View{0, a.W.scale, a.W.shift, a.W.C};
    const int i = inst_of(a.I, g);
    return View{__ldg(a.I.delta + i), __ldg(a.I.scale + i), __ldg(a.I.shift + i), __ldg(a.I.C + i)};
}

// Whether credit g belongs to an instance this launch works on.
template <bool MULTI, typename T>
__device__ __forceinline__ bool in_active(const Args<T> &a, int g) {
    if (!MULTI || !a.I.active) return true;
    return __ldg(a.I.active + inst_of(a.I, g)) != 0;
}

// View of a lane that holds no entry.  It must still be the instance's view
// when there is one instance: such a lane processes edges of other lanes'
// entries, and with one instance views are not exchanged between lanes.
template <bool MULTI, typename T>
__device__ __forceinline__ View idle_view(const Args<T> &a) {
    return MULTI ? View{0, 0, 0, 0} : View{0, a.W.scale, a.W.shift, a.W.C};
}

template <bool MULTI>
__device__ __forceinline__ View shfl_view(const View &v, int j) {
    if (!MULTI) return v;
    return View{__shfl_sync(FULL, v.delta, j), __shfl_sync(FULL, v.scale, j), __shfl_sync(FULL, v.shift, j),
                __shfl_sync(FULL, v.C, j)};
}

// ---------------------------------------------------------------------------
// Bound C = M_G = sum_v max(0, max_e -w'(e)) and max |w'| (Sec. 3.1), from the
// per-vertex extremes of the weights: O(n), coalesced.
__global__ void k_bound(DevArena A, WeightView W, unsigned long long *out_C, unsigned long long *out_wmax) {
    long long sum = 0, wmax = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        const int lo = __ldg(A.wmin + v), hi = __ldg(A.wmax + v);
        const long long mn = wmap_min(lo, hi, W), mx = wmap_max(lo, hi, W);
        sum += mn < 0 ? -mn : 0;
        wmax = max(wmax, max(mn < 0 ? -mn : mn, mx < 0 ? -mx : mx));
    }
    for (int d = 16; d; d >>= 1) {
        sum += __shfl_down_sync(FULL, sum, d);
        wmax = max(wmax, __shfl_down_sync(FULL, wmax, d));
    }
    if (lane_id() == 0) {
        atomicAdd(out_C, (unsigned long long)sum);
        atomicMax(out_wmax, (unsigned long long)wmax);
    }
}

template <typename T>
__global__ void k_fill(T *p, long long n, T v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// Tiles of an O(n) pass (warm start, init, sweeps, proofs, counts): warps
// take 32-credit tiles in order.  A batched lift of the certified trials
// works on few instances; its launches carry the ascending list of the tiles
// that cover those instances, and the passes visit only these.  Lanes of
// other instances in a boundary tile are skipped as everywhere else.
__device__ __forceinline__ long long tile_count(const int *tiles, long long ntiles, int g0, int g1) {
    return tiles ? ntiles : ((long long)(g1 - g0) + 31) / 32;
}
__device__ __forceinline__ int tile_base(const int *tiles, long long t, int g0) {
    return tiles ? (__ldg(tiles + t) << 5) : g0 + (int)(t << 5);
}

// ---------------------------------------------------------------------------
// Warm start.  A player-1 vertex u on a cycle of player-1 vertices whose
// weight (under the weight view) is negative is won by player 1: player 1
// can keep the play on that cycle forever, so every credit runs out
// (Lemma "EGcycles" with memoryless determinacy, Sec. 3).  Its least-EPM
// value is TOP, so starting it at TOP stays below the least fixpoint.
// Looked for: negative self-loops and 2-cycles u -> t -> u with t a player-1
// vertex, by comparing each out-edge (u, t) with each in-edge (s, u) for
// s == t.  A vertex with at most SEED_LANE_EDGES in- and out-edges together
// is checked by one lane alone, over its own rows; a larger one by the whole
// warp.  Vertices with out-degree x in-degree above max_pairs are skipped
// (the warm start is optional, missing a cycle only costs time).
constexpr int SEED_LANE_EDGES = 64;

template <bool MULTI, typename T>
__global__ void k_seed(Args<T> a, long long max_pairs, unsigned *seed_bits, unsigned long long *count, int g0,
                       int g1) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned found_total = 0;
    const long long ntiles = tile_count(a.tiles, a.ntiles, g0, g1);
    for (long long t = gw; t < ntiles; t += nw) {
        const int g = tile_base(a.tiles, t, g0) + lane;
        bool mine = false;  // a player-1 credit of this lane, within max_pairs
        View vw = idle_view<MULTI>(a);
        int u = 0, ob = 0, oe = 0, ib = 0, ie = 0;
        if (g < g1 && in_active<MULTI>(a, g)) {
            vw = view_of<MULTI>(a, g);
            u = g - vw.delta;
            if (((__ldg(A.owner_bits + (u >> 5)) >> (u & 31)) & 1u) ^ a.inv) {
                ob = __ldg(A.row_ptr + u);
                oe = __ldg(A.row_ptr + u + 1);
                ib = __ldg(A.rrow_ptr + u);
                ie = __ldg(A.rrow_ptr + u + 1);
                mine = (long long)(oe - ob) * (long long)(ie - ib) <= max_pairs;
            }
        }
        const bool small = mine && (oe - ob) + (ie - ib) <= SEED_LANE_EDGES;
        bool found = false;
        if (small) {
            // the lane alone: a 128-bit filter of its player-1 predecessors
            // (two bits per id, from its low and next 7 bits) rejects almost
            // every out-edge with one test; the in-row is searched only
            // where the filter matches
            unsigned long long filt[2] = {0, 0};
#pragma unroll 4
            for (int j = ib; j < ie; ++j) {
                const unsigned sj = __ldg(A.rcol + j);
                if (((sj & P1_FLAG) != 0) != (a.inv != 0)) {
                    const unsigned h1 = sj & 127u, h2 = (sj >> 7) & 127u;
                    filt[h1 >> 6] |= 1ull << (h1 & 63u);
                    filt[h2 >> 6] |= 1ull << (h2 & 63u);
                }
            }
#pragma unroll 4
            for (int k = ob; k < oe; ++k) {
                const int t = __ldg(A.col + k);
                const unsigned h1 = (unsigned)t & 127u, h2 = ((unsigned)t >> 7) & 127u;
                const bool maybe = ((filt[h1 >> 6] >> (h1 & 63u)) & 1ull) && ((filt[h2 >> 6] >> (h2 & 63u)) & 1ull);
                if (t == u) {
                    if (wmapv(__ldg(A.w + k), vw) < 0) found = true;  // negative self-loop
                } else if (maybe) {
                    const long long wt = wmapv(__ldg(A.w + k), vw);
                    for (int j = ib; j < ie; ++j) {
                        const unsigned sj = __ldg(A.rcol + j);
                        if ((int)(sj & 0x7fffffffu) == t && ((sj & P1_FLAG) != 0) != (a.inv != 0) &&
                            wt + wmapv(__ldg(A.rw + j), vw) < 0)
                            found = true;
                    }
                }
            }
        }
        // the larger ones, one at a time by the whole warp
        unsigned big = __ballot_sync(FULL, mine && !small);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int bu = __shfl_sync(FULL, u, src);
            const int bob = __shfl_sync(FULL, ob, src), boe = __shfl_sync(FULL, oe, src);
            const int bib = __shfl_sync(FULL, ib, src), bie = __shfl_sync(FULL, ie, src);
            const View bv = shfl_view<MULTI>(vw, src);
            bool bfound = false;
            for (int kb = bob; kb < boe; kb += 32) {
                const int k = kb + lane;
                int t = -1;
                long long wt = 0;
                if (k < boe) {
                    t = __ldg(A.col + k);
                    wt = wmapv(__ldg(A.w + k), bv);
                    if (t == bu && wt < 0) bfound = true;  // negative self-loop
                }
                for (int jb = bib; jb < bie; jb += 32) {
                    const int j = jb + lane;
                    unsigned sj = 0;
                    long long wj = 0;
                    if (j < bie) {
                        sj = __ldg(A.rcol + j);
                        wj = wmapv(__ldg(A.rw + j), bv);
                    }
                    const int cnt = min(32, bie - jb);
                    for (int q = 0; q < cnt; ++q) {
                        const unsigned sq = __shfl_sync(FULL, sj, q);
                        const long long wq = __shfl_sync(FULL, wj, q);
                        if (((sq & P1_FLAG) != 0) != (a.inv != 0) && (int)(sq & 0x7fffffffu) == t && t != bu &&
                            wt + wq < 0)
                            bfound = true;
                    }
                }
            }
            if (__any_sync(FULL, bfound) && lane == src) found = true;
        }
        if (found) {
            atomicOr(seed_bits + (g >> 5), 1u << (g & 31));
            ++found_total;
        }
    }
    for (int d = 16; d; d >>= 1) found_total += __shfl_down_sync(FULL, found_total, d);
    if (lane == 0 && found_total) atomicAdd(count, (unsigned long long)found_total);
}

// ---------------------------------------------------------------------------
// Initialisation (Algorithm 3's set-up of f and of the first frontier, with
// the first lift folded in):
// f(v) = delta(0, v)(v).  With every successor at 0 that is max(0, -w') taken
// at the smallest w' of v's edges for a player-1 vertex (max over edges) and
// at the largest for a player-0 vertex (min over edges), so it needs only the
// per-vertex weight extremes.  It is positive exactly for the initial set L of
// Algorithm 1 (V0 with every edge negative, V1 with some edge negative); those
// vertices, and the warm-start ones (TOP), enter the push list of the first
// round (list counter `slot`, buffer `buf`).  Credits [g0, g1) are set.
template <bool MULTI, typename T>
__global__ void __launch_bounds__(THREADS) k_init(Args<T> a, int g0, int g1, int slot, int buf, int list) {
    const DevArena &A = a.A;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const long long ntiles = tile_count(a.tiles, a.ntiles, g0, g1);
    for (long long t = gw; t < ntiles; t += nw) {
        const int g = tile_base(a.tiles, t, g0) + lane_id();
        bool want = false;
        int work = 0;
        if (g < g1 && in_active<MULTI>(a, g)) {
            const View vw = view_of<MULTI>(a, g);
            const int v = g - vw.delta;
            const bool p1 = ((__ldg(A.owner_bits + (v >> 5)) >> (v & 31)) & 1u) ^ a.inv;
            const bool fz = a.frozen && ((__ldg(a.frozen + (g >> 5)) >> (g & 31)) & 1u);
            T f0;
            if (fz) {
                f0 = T(0);
            } else if (a.seed_bits && ((a.seed_bits[g >> 5] >> (g & 31)) & 1u)) {
                f0 = Cred<T>::TOP;
            } else {
                const int lo = __ldg(A.wmin + v), hi = __ldg(A.wmax + v);
                const long long smin = vw.scale >= 0 ? wmapv(lo, vw) : wmapv(hi, vw);
                const long long smax = vw.scale >= 0 ? wmapv(hi, vw) : wmapv(lo, vw);
                f0 = ominus<T>(T(0), p1 ? smin : smax, vw.C);
            }
            a.f[g] = f0;
            work = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
            want = !fz && f0 > T(0) && work > 0;
        }
        warp_append(list && want, (unsigned)g, work, &a.ctrl->push_ctr[slot], a.push_items[buf], a.push_offs[buf]);
    }
}

// First lift of the vertices of one topological level of an SCC-ordered
// solve: the lift over all successors with the current credits (the lower
// levels are final, this level's vertices start at 0 or, warm-started, at
// TOP); a vertex whose credit is positive joins the push list of round 0.
// Reads of other vertices of the level may see their old or new credit:
// both are at or below the least fixpoint.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_init_level(Args<T> a, int level) {
    const DevArena &A = a.A;
    const int nthreads = gridDim.x * blockDim.x;
    const WeightView &W = a.W;
    for (int base = blockIdx.x * blockDim.x; base < A.n; base += nthreads) {
        const int v = base + threadIdx.x;
        bool want = false;
        int work = 0;
        if (v < A.n && __ldg(a.level + v) == level) {
            const bool p1 = ((__ldg(A.owner_bits + (v >> 5)) >> (v & 31)) & 1u) ^ a.inv;
            T cur = ld_cg(a.f + v);
            if (cur != Cred<T>::TOP) {
                T g = p1 ? T(0) : Cred<T>::TOP;
                for (int e = __ldg(A.row_ptr + v); e < __ldg(A.row_ptr + v + 1); ++e) {
                    const T t = ominus<T>(ld_cg(a.f + __ldg(A.col + e)), wmap(__ldg(A.w + e), W), W.C);
                    g = p1 ? max(g, t) : min(g, t);
                }
                if (g > cur) {
                    atomicMax(a.f + v, g);
                    cur = g;
                }
            }
            work = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
            want = cur > T(0) && work > 0;
        }
        warp_append(want, (unsigned)v, work, &a.ctrl->push_ctr[0], a.push_items[0], a.push_offs[0]);
    }
}

// Credits of an SCC-ordered solve before its first level: TOP on the warm
// start's vertices, else 0.
template <typename T>
__global__ void k_level_start(T *f, int n, const unsigned *seed_bits) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        f[v] = seed_bits && ((seed_bits[v >> 5] >> (v & 31)) & 1u) ? Cred<T>::TOP : T(0);
}

// Per-instance bound C = M_G and max |w'| of every instance (one credit per
// thread, from the weight extremes of its arena vertex; a warp whose credits
// all belong to one instance adds them with one atomic).
__global__ void k_bound_inst(DevArena A, InstTable I, int nf, unsigned long long *C, unsigned long long *wmax) {
    const int lane = lane_id();
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < nf; base += gridDim.x * blockDim.x) {
        const int g = base + lane;
        int i = -1;
        long long def = 0, mag = 0;
        if (g < nf) {
            i = inst_of(I, g);
            const View vw{__ldg(I.delta + i), __ldg(I.scale + i), __ldg(I.shift + i), 0};
            const int v = g - vw.delta;
            const int lo = __ldg(A.wmin + v), hi = __ldg(A.wmax + v);
            const long long a1 = wmapv(lo, vw), a2 = wmapv(hi, vw);
            const long long mn = min(a1, a2), mx = max(a1, a2);
            def = mn < 0 ? -mn : 0;
            mag = max(mn < 0 ? -mn : mn, mx < 0 ? -mx : mx);
        }
        const int i0 = __shfl_sync(FULL, i, 0);
        if (__all_sync(FULL, i == i0)) {
            for (int d = 16; d; d >>= 1) {
                def += __shfl_down_sync(FULL, def, d);
                mag = max(mag, __shfl_down_sync(FULL, mag, d));
            }
            if (lane == 0 && i0 >= 0) {
                atomicAdd(C + i0, (unsigned long long)def);
                atomicMax(wmax + i0, (unsigned long long)mag);
            }
        } else if (i >= 0) {
            atomicAdd(C + i, (unsigned long long)def);
            atomicMax(wmax + i, (unsigned long long)mag);
        }
    }
}

// ---------------------------------------------------------------------------
// Window helpers.  A warp works on up to 32 list entries at a time, one per
// lane; lane j holds its entry's first edge `beg` and the entry's offset `o`
// in the warp's edge coordinates (non-decreasing over lanes; lanes without an
// entry hold the window total).  Edge x belongs to the largest j with o_j <= x.

__device__ __forceinline__ int owner_lane(int o, int xl) {
    int j = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int oj = __shfl_sync(FULL, o, j + s);
        if (oj <= xl) j += s;
    }
    return j;
}

// Exclusive warp scan of per-lane works; returns the total.
__device__ __forceinline__ int warp_exclusive(int work, int &excl) {
    const int lane = lane_id();
    int incl = work;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
    }
    excl = incl - work;
    return __shfl_sync(FULL, incl, 31);
}

// Minimum of f(u) (-) w(v,u) over the edges [x0, stop) of the window, per
// owning lane (TOP for lanes that own none of them).  vw: the lane's view.
template <bool MULTI, typename T>
__device__ __forceinline__ T pull_min(const Args<T> &a, int beg, int o, const View &vw, int x0, int stop, T *red) {
    const int lane = lane_id();
    red[lane] = Cred<T>::TOP;
    __syncwarp();
    for (int xb = x0; xb < stop; xb += 32) {
        const int xl = xb + lane;
        const bool act = xl < stop;
        const int j = owner_lane(o, xl);
        const int bj = __shfl_sync(FULL, beg, j);
        const int oj = __shfl_sync(FULL, o, j);
        const View vj = shfl_view<MULTI>(vw, j);
        T t = Cred<T>::TOP;
        if (act) {
            const int e = bj + (xl - oj);
            const int u = __ldg(a.A.col + e) + vj.delta;
            t = ominus<T>(ld_cg(a.f + u), wmapv(__ldg(a.A.w + e), vj), vj.C);
        }
        const int key = act ? j : 32 + lane;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T ov = __shfl_up_sync(FULL, t, d);
            const int ok = __shfl_up_sync(FULL, key, d);
            if (lane >= d && ok == key) t = min(t, ov);
        }
        const int nk = __shfl_down_sync(FULL, key, 1);
        if (act && (lane == 31 || nk != key)) red[j] = min(red[j], t);
        __syncwarp();
    }
    const T g = red[lane];
    __syncwarp();
    return g;
}

// ---------------------------------------------------------------------------
// Dense sweeps before the worklist rounds.  One sweep evaluates the lift
// delta(f, v) of every credit in index order and raises f(v) to it in place:
// the minimum over v's edges of f(u) (-) w(v, u) for a player-0 vertex, the
// maximum for a player-1 vertex (Sec. 3.1).  Each credit has a single writer
// (its lane), so no atomics are needed, and a warp reads 32 consecutive rows
// with coalesced loads.  The lift is monotone, so raising credits to it from
// below, with successor credits read old or new, never passes the least
// fixpoint (the chaotic iteration of Sec. 3.1's lifting).
//
// Only the last sweep builds the first round's push list: a credit it raised
// joins the list.  A credit whose lift read a successor before that
// successor rose in the last sweep has the successor on the list, and one
// that read it before a rise in an earlier sweep read it again in a later
// sweep; so after the rounds that follow, every credit is its own lift.
// Warm-start credits at TOP and frozen credits (held at 0) are left alone.

// Per owning lane, the lift over the warp's edges [0, stop): the minimum of
// f(u) (-) w for a player-0 entry, the maximum for a player-1 entry (lanes
// owning no edge get TOP or 0).  beg, o, vw as in pull_min; p1: the lane's
// entry belongs to player 1.
template <bool MULTI, typename T>
__device__ __forceinline__ T sweep_lift(const Args<T> &a, int beg, int o, const View &vw, bool p1, int stop,
                                        T *red) {
    const int lane = lane_id();
    red[lane] = p1 ? T(0) : Cred<T>::TOP;
    __syncwarp();
    for (int xb = 0; xb < stop; xb += 32) {
        const int xl = xb + lane;
        const bool act = xl < stop;
        const int j = owner_lane(o, xl);
        const int bj = __shfl_sync(FULL, beg, j);
        const int oj = __shfl_sync(FULL, o, j);
        const bool pj = __shfl_sync(FULL, p1, j);
        const View vj = shfl_view<MULTI>(vw, j);
        T t = pj ? T(0) : Cred<T>::TOP;
        if (act) {
            const int e = bj + (xl - oj);
            const int u = __ldg(a.A.col + e) + vj.delta;
            t = ominus<T>(ld_cg(a.f + u), wmapv(__ldg(a.A.w + e), vj), vj.C);
        }
        const int key = act ? j : 32 + lane;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T ov = __shfl_up_sync(FULL, t, d);
            const int ok = __shfl_up_sync(FULL, key, d);
            if (lane >= d && ok == key) t = pj ? max(t, ov) : min(t, ov);
        }
        const int nk = __shfl_down_sync(FULL, key, 1);
        if (act && (lane == 31 || nk != key)) red[j] = pj ? max(red[j], t) : min(red[j], t);
        __syncwarp();
    }
    const T g = red[lane];
    __syncwarp();
    return g;
}

// Rows of at most this many edges are walked by one lane in a sweep.
constexpr int SWEEP_LANE_DEG = 32;

// One sweep over the credits [0, nf); with `last`, raised credits join the
// push list of round 0 (list counter 0, buffer 0).
template <bool MULTI, typename T>
__global__ void __launch_bounds__(THREADS) k_sweep(Args<T> a, int last) {
    __shared__ T red_all[WARPS][32];
    T *red = red_all[threadIdx.x >> 5];
    const DevArena &A = a.A;
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long relax = 0, lifts = 0;
    const long long ntiles = tile_count(a.tiles, a.ntiles, 0, a.nf);
    for (long long t = gw; t < ntiles; t += nw) {
        const int g = tile_base(a.tiles, t, 0) + lane;
        bool on = g < a.nf && in_active<MULTI>(a, g);
        View vw = idle_view<MULTI>(a);
        bool p1 = false;
        int v = 0, beg = 0, work = 0;
        T cur = T(0);
        if (on) {
            vw = view_of<MULTI>(a, g);
            v = g - vw.delta;
            const bool fz = a.frozen && ((__ldg(a.frozen + (g >> 5)) >> (g & 31)) & 1u);
            cur = ld_cg(a.f + g);
            on = !fz && cur != Cred<T>::TOP && vw.C >= 0;
            p1 = ((__ldg(A.owner_bits + (v >> 5)) >> (v & 31)) & 1u) ^ a.inv;
            if (on) {
                beg = __ldg(A.row_ptr + v);
                work = __ldg(A.row_ptr + v + 1) - beg;
            }
        }
        // a light row is walked by its own lane (the rows of neighbouring
        // credits share cache lines, and lanes exchange nothing); the heavy
        // rows of the warp are walked by all its lanes together
        const bool light = work <= SWEEP_LANE_DEG;
        T res = p1 ? T(0) : Cred<T>::TOP;
        if (light) {
            const int *cp = A.col + beg;
            const int *wp = A.w + beg;
#pragma unroll 4
            for (int k = 0; k < work; ++k) {
                const T t = ominus<T>(ld_cg(a.f + (__ldg(cp + k) + vw.delta)), wmapv(__ldg(wp + k), vw), vw.C);
                res = p1 ? max(res, t) : min(res, t);
            }
        }
        int o;
        const int heavy = warp_exclusive(light ? 0 : work, o);
        if (heavy > 0) {
            const T hr = sweep_lift<MULTI, T>(a, beg, o, vw, p1, heavy, red);
            if (!light) res = hr;
        }
        bool rose = false;
        if (work > 0 && res > cur) {
            st_cg(a.f + g, res);
            rose = true;
        }
        relax += __reduce_add_sync(FULL, (unsigned)work);
        lifts += __popc(__ballot_sync(FULL, work > 0 && !p1));
        if (last) {
            const int pwork = rose ? __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v) : 0;
            warp_append(rose && pwork > 0, (unsigned)g, pwork, &a.ctrl->push_ctr[0], a.push_items[0],
                        a.push_offs[0]);
        }
    }
    if (lane == 0 && relax) {
        atomicAdd(&a.ctrl->relax, relax);
        atomicAdd(&a.ctrl->lifts, lifts);
    }
}

// Per-warp staging of list appends: entries collect in shared memory and
// reach the global list (items, offs, packed counter) with one atomic per
// flush instead of one per warp step, which keeps the counters -- shared by
// every warp of the grid -- out of the critical path.
constexpr int STAGE = 128;

struct Stager {
    int *item;  // STAGE entries in shared memory
    int *work;
    int n;      // warp-uniform fill
    unsigned long long *ctr;
    int *items;
    int *offs;
};

__device__ __forceinline__ void stage_flush(Stager &S) {
    if (S.n == 0) return;
    __syncwarp();
    const int lane = lane_id();
    constexpr int PER = STAGE / 32;
    const int b = lane * PER;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (b + k < S.n) sum += S.work[b + k];
    int excl;
    const int total = warp_exclusive(sum, excl);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(S.ctr, ((unsigned long long)(unsigned)total << 32) | (unsigned)S.n);
    base = __shfl_sync(FULL, base, 0);
    const unsigned bi = (unsigned)(base & 0xffffffffu);
    int off = (int)(base >> 32) + excl;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (b + k < S.n) {
            S.items[bi + b + k] = S.item[b + k];
            S.offs[bi + b + k] = off;
            off += S.work[b + k];
        }
    }
    __syncwarp();
    S.n = 0;
}

// Warp-aggregated append through the stage.  Called by all 32 lanes.
__device__ __forceinline__ void stage_append(Stager &S, bool want, unsigned item, int work) {
    const unsigned mask = __ballot_sync(FULL, want);
    if (mask == 0) return;
    const int k = __popc(mask);
    if (S.n + k > STAGE) stage_flush(S);
    if (want) {
        const int at = S.n + __popc(mask & ((1u << lane_id()) - 1u));
        S.item[at] = (int)item;
        S.work[at] = work;
    }
    S.n += k;
    __syncwarp();
}

// Per-warp state of one round's push phase: the local worklist (a stack in
// shared memory), the staged appends to the next round's lists, and
// counters of the work done through the local worklist.
template <typename T>
struct Local {
    int *stack;
    int top;
    bool on;
    Stager next_pull, next_push;
    unsigned long long relax, lifts, pushes;
};

constexpr unsigned NEED_NONE = 0, NEED_PULL = 1, NEED_PUSH = 2;

// Routes credits that need work in this or the next round.  NEED_PULL: a
// player-0 vertex that may lift; NEED_PUSH: a vertex whose rise must reach
// its predecessors.  The next round's bitmap of that kind marks a credit as
// queued -- in some warp's local worklist or in the next round's list -- so a
// credit already queued absorbs the request (it reads fresh credits when it
// is processed).  Newly queued small vertices go to the warp's local
// worklist while it has room; the rest join the next round's lists.
template <typename T>
__device__ __forceinline__ void route(const Args<T> &a, int r, unsigned need, int p, int work, Local<T> &L) {
    const int lane = lane_id();
    bool fresh = false;
    if (need != NEED_NONE) {
        unsigned *bits = need == NEED_PULL ? a.bits_pull[(r + 1) & 1] : a.bits_push[(r + 1) & 1];
        const unsigned bit = 1u << (p & 31);
        fresh = !(atom_or_release(bits + (p >> 5), bit) & bit);
    }
    const bool local_ok = fresh && L.on && work <= a.local_maxdeg;
    const unsigned lm = __ballot_sync(FULL, local_ok);
    const int rank = __popc(lm & ((1u << lane) - 1u));
    const int room = LOCAL_CAP - L.top;
    bool placed = false;
    if (local_ok && rank < room) {
        L.stack[L.top + rank] = p | (need == NEED_PUSH ? (int)P1_FLAG : 0);
        placed = true;
    }
    L.top += min(__popc(lm), room);
    const bool gpull = fresh && !placed && need == NEED_PULL;
    const bool gpush = fresh && !placed && need == NEED_PUSH;
    stage_append(L.next_pull, gpull, (unsigned)p, work);
    stage_append(L.next_push, gpush, (unsigned)p, work);
}

// Sends the values `val` of the window's entries over their in-edges
// [x0, stop): t = val (-) w(p, v) for every predecessor p.  A player-1 p takes
// max(f(p), t) (atomicMax) and, if it rose, needs a push; a player-0 p with
// f(p) < t may need a lift.
template <bool MULTI, typename T>
__device__ __forceinline__ void push_edges(const Args<T> &a, int r, int beg, int o, T val, const View &vw, int x0,
                                           int stop, Local<T> &L) {
    const int lane = lane_id();
    for (int xb = x0; xb < stop; xb += 32) {
        const int xl = xb + lane;
        const bool act = xl < stop;
        const int j = owner_lane(o, xl);
        const int bj = __shfl_sync(FULL, beg, j);
        const int oj = __shfl_sync(FULL, o, j);
        const T vj = __shfl_sync(FULL, val, j);
        const View wj = shfl_view<MULTI>(vw, j);
        unsigned need = NEED_NONE;
        int p = 0, work = 0;
        if (act && wj.C >= 0) {
            const int e = bj + (xl - oj);
            const unsigned pr = __ldg(a.A.rcol + e);
            const int pa = (int)(pr & 0x7fffffffu);
            p = pa + wj.delta;
            const bool p1 = ((pr & P1_FLAG) != 0) != (a.inv != 0);
            // the row the predecessor would be queued with (in-edges for a
            // player-1 rise, out-edges for a player-0 lift), loaded beside
            // its credit rather than after the test
            const int *rp = p1 ? a.A.rrow_ptr : a.A.row_ptr;
            const int rb = __ldg(rp + pa), re = __ldg(rp + pa + 1);
            const bool fz = (a.frozen && ((__ldg(a.frozen + (p >> 5)) >> (p & 31)) & 1u)) ||
                            (a.level && __ldg(a.level + p) > a.cur_level);
            const T t = ominus<T>(vj, wmapv(__ldg(a.A.rw + e), wj), wj.C);
            if (!fz && t > ld_cg(a.f + p)) {
                if (p1) {
                    if (t > atomicMax(a.f + p, t)) {
                        work = re - rb;
                        if (work > 0) need = NEED_PUSH;
                    }
                } else {
                    work = re - rb;
                    need = NEED_PULL;
                }
            }
        }
        route<T>(a, r, need, p, work, L);
    }
}

// Empties the warp's local worklist: windows of up to 32 entries, each a
// lift of its player-0 entries (in place, atomicMax) followed by a push of
// every entry that rose and of the player-1 entries.  Runs for at most
// a.local_windows windows, then hands what is left to the next round.
template <bool MULTI, typename T>
__device__ void drain_local(const Args<T> &a, int r, T *red, Local<T> &L) {
    const int lane = lane_id();
    int windows = 0;
    while (L.top > 0) {
        if (windows >= a.local_windows) L.on = false;
        ++windows;
        const int take = min(32, L.top);
        bool have = lane < take;
        const int raw = have ? L.stack[L.top - 1 - lane] : 0;
        __syncwarp();
        L.top -= take;
        const int g = raw & 0x7fffffff;
        View vw = idle_view<MULTI>(a);
        if (have) vw = view_of<MULTI>(a, g);
        if (have && vw.C < 0) {  // retired instance: unmark and drop
            atomicAnd(((raw & (int)P1_FLAG) ? a.bits_push[(r + 1) & 1] : a.bits_pull[(r + 1) & 1]) + (g >> 5),
                      ~(1u << (g & 31)));
            have = false;
            vw = idle_view<MULTI>(a);
        }
        const bool is_push = have && (raw & (int)P1_FLAG);
        const bool is_pull = have && !(raw & (int)P1_FLAG);
        const int v = g - vw.delta;
        // both rows of the entry up front: they do not depend on credits, so
        // these loads need not wait for the unmark below, and the push after
        // a lift finds its row already loaded
        int pbeg = 0, pwork = 0, rbeg = 0, rwork = 0;
        if (is_pull) {
            pbeg = __ldg(a.A.row_ptr + v);
            pwork = __ldg(a.A.row_ptr + v + 1) - pbeg;
        }
        if (have) {
            rbeg = __ldg(a.A.rrow_ptr + v);
            rwork = __ldg(a.A.rrow_ptr + v + 1) - rbeg;
        }
        if (!L.on) {  // budget spent: the entries (still marked) join the next round's lists
            const int work = is_pull ? pwork : rwork;
            stage_append(L.next_pull, is_pull, (unsigned)g, work);
            stage_append(L.next_push, is_push, (unsigned)g, work);
            continue;
        }
        if (have) {  // unmark before reading credits
            unsigned *bits = is_pull ? a.bits_pull[(r + 1) & 1] : a.bits_push[(r + 1) & 1];
            atom_and_acquire(bits + (g >> 5), ~(1u << (g & 31)));
        }
        // lifts
        int po;
        const int ptotal = warp_exclusive(pwork, po);
        T gmin = Cred<T>::TOP;
        if (ptotal > 0) gmin = pull_min<MULTI, T>(a, pbeg, po, vw, 0, ptotal, red);
        bool rose = is_push;
        T val = T(0);
        if (is_pull) {
            rose = gmin > atomicMax(a.f + g, gmin);
            val = gmin;
        } else if (is_push) {
            val = ld_cg(a.f + g);
        }
        L.relax += ptotal;
        L.lifts += __popc(__ballot_sync(FULL, is_pull));
        // pushes: small ones here, large ones to the next round
        int qbeg = 0, qwork = 0;
        if (rose) {
            qbeg = rbeg;
            qwork = rwork;
        }
        const bool big = rose && qwork > a.local_maxdeg;
        {
            bool gpush = false;
            if (big) {
                const unsigned bit = 1u << (g & 31);
                gpush = !(atom_or_release(a.bits_push[(r + 1) & 1] + (g >> 5), bit) & bit);
            }
            stage_append(L.next_push, gpush, (unsigned)g, qwork);
        }
        if (big || !rose) qwork = 0;
        int qo;
        const int qtotal = warp_exclusive(qwork, qo);
        if (qtotal > 0) push_edges<MULTI, T>(a, r, qbeg, qo, val, vw, 0, qtotal, L);
        L.relax += qtotal;
        L.pushes += __popc(__ballot_sync(FULL, qwork > 0));
    }
}

// ---------------------------------------------------------------------------
// Work split of a round's list over the warps, in its edge coordinates
// [0, total).  A list of at most `chunk` edges per warp is cut into one equal
// piece per warp.  A longer one is cut into chunks of `chunk` edges that the
// warps take in order, the first by warp id and the rest from the round's
// take counter, so that the whole grid sweeps the list together: the credits
// and rows its gathers reach (those of the vertices near the sweep, which in
// a list built in vertex order are the same few games) stay in L2, where
// with one piece per warp every warp would pull its own far part of the arena
// through L2 at once.
struct ChunkPlan {
    long long first;   // the warp's first chunk
    long long K;       // edges per chunk
    long long nwarps;  // chunks handed out by warp id
    bool dyn;          // further chunks come from the take counter
};

__device__ __forceinline__ ChunkPlan chunk_plan(int total, int chunk) {
    ChunkPlan cp;
    cp.nwarps = (long long)gridDim.x * WARPS;
    cp.first = (long long)blockIdx.x * WARPS + (threadIdx.x >> 5);
    cp.dyn = chunk > 0 && (long long)total > cp.nwarps * chunk;
    cp.K = cp.dyn ? max(chunk, 32) : max(32LL, ((long long)total + cp.nwarps - 1) / cp.nwarps);
    return cp;
}

// The warp's next chunk; with the static split one past every list.
__device__ __forceinline__ long long next_chunk(const ChunkPlan &cp, unsigned *take) {
    if (!cp.dyn) return (long long)INT_MAX;
    unsigned t = 0;
    if (lane_id() == 0) t = atomicAdd(take, 1u);
    return cp.nwarps + (long long)__shfl_sync(FULL, t, 0);
}

// ---------------------------------------------------------------------------
// Pull phase: lift the player-0 vertices of the pull list of round r.
template <bool MULTI, typename T>
__device__ void pull_phase(const Args<T> &a, int r, T *red, Stager &out) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const unsigned long long ctr = ld_cg(&a.ctrl->pull_ctr[r % 3]);
    const int cnt = (int)(ctr & 0xffffffffu);
    const int total = (int)(ctr >> 32);
    const int *items = a.pull_items[r & 1];
    const int *offs = a.pull_offs[r & 1];
    unsigned *bits = a.bits_pull[r & 1];
    unsigned *bits_q = a.bits_push[r & 1];

    const ChunkPlan cp = chunk_plan(total, a.chunk);
    for (long long c = cp.first; c * cp.K < total; c = next_chunk(cp, &a.ctrl->pull_take[r % 3])) {
        const int lo = (int)(c * cp.K);
        const int hi = (int)min((long long)total, c * cp.K + cp.K);
        int i = warp_find(offs, cnt, lo);
        int x = lo;
        while (x < hi) {
            const int ii = i + lane;
            const bool valid = ii < cnt;
            int g = 0, v = 0, o = total, oend = total, beg = 0;
            View vw = idle_view<MULTI>(a);
            if (valid) {
                g = ld_cg(items + ii) & 0x7fffffff;
                vw = view_of<MULTI>(a, g);
                v = g - vw.delta;
                o = ld_cg(offs + ii);
                oend = ii + 1 < cnt ? ld_cg(offs + ii + 1) : total;
                beg = __ldg(A.row_ptr + v);
            }
            const int stop = min(hi, __shfl_sync(FULL, oend, 31));
            const T gmin = pull_min<MULTI, T>(a, beg, o, vw, x, stop, red);
            // finish the lifts of this window's entries
            bool changed = false;
            int pwork = 0;
            if (valid && o < stop && oend > x) {
                if (o >= lo) atomicAnd(bits + (g >> 5), ~(1u << (g & 31)));  // consumed
                const int seen = min(oend, stop) - max(o, x);
                T res = gmin;
                bool done = true;
                if (seen != oend - o) {  // lift split across chunks: merge partial minima
                    atomicMin(a.acc + g, gmin);
                    __threadfence();
                    const int before = atomicAdd(a.acc_done + g, seen);
                    done = before + seen == oend - o;
                    if (done) {
                        __threadfence();
                        res = xchg(a.acc + g, Cred<T>::TOP);
                        atomicExch(a.acc_done + g, 0);
                    }
                }
                if (done && vw.C >= 0 && res > ld_cg(a.f + g) && res > atomicMax(a.f + g, res)) {
                    pwork = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
                    if (pwork > 0) {
                        const unsigned bit = 1u << (g & 31);
                        changed = !(ld_cg(bits_q + (g >> 5)) & bit) && !(atomicOr(bits_q + (g >> 5), bit) & bit);
                    }
                }
            }
            stage_append(out, changed, (unsigned)g, pwork);
            x = stop;
            i += 32;
        }
    }
}

// ---------------------------------------------------------------------------
// Push phase: send the rises of the push list of round r to predecessors,
// then work through the warp's local worklist.
template <bool MULTI, typename T>
__device__ void push_phase(const Args<T> &a, int r, T *red, Local<T> &L) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const unsigned long long ctr = ld_cg(&a.ctrl->push_ctr[r % 3]);
    const int cnt = (int)(ctr & 0xffffffffu);
    const int total = (int)(ctr >> 32);
    const int *items = a.push_items[r & 1];
    const int *offs = a.push_offs[r & 1];
    unsigned *bits_cur = a.bits_push[r & 1];

    L.top = 0;
    L.on = a.local_windows > 0;
    L.next_pull.n = 0;
    L.next_pull.ctr = &a.ctrl->pull_ctr[(r + 1) % 3];
    L.next_pull.items = a.pull_items[(r + 1) & 1];
    L.next_pull.offs = a.pull_offs[(r + 1) & 1];
    L.next_push.n = 0;
    L.next_push.ctr = &a.ctrl->push_ctr[(r + 1) % 3];
    L.next_push.items = a.push_items[(r + 1) & 1];
    L.next_push.offs = a.push_offs[(r + 1) & 1];
    const ChunkPlan cp = chunk_plan(total, a.chunk);
    for (long long c = cp.first; c * cp.K < total; c = next_chunk(cp, &a.ctrl->push_take[r % 3])) {
        const int lo = (int)(c * cp.K);
        const int hi = (int)min((long long)total, c * cp.K + cp.K);
        int i = warp_find(offs, cnt, lo);
        int x = lo;
        while (x < hi) {
            const int ii = i + lane;
            const bool valid = ii < cnt;
            int o = total, oend = total, beg = 0;
            T val = T(0);
            View vw = idle_view<MULTI>(a);
            if (valid) {
                const int g = ld_cg(items + ii) & 0x7fffffff;
                vw = view_of<MULTI>(a, g);
                const int v = g - vw.delta;
                o = ld_cg(offs + ii);
                oend = ii + 1 < cnt ? ld_cg(offs + ii + 1) : total;
                beg = __ldg(A.rrow_ptr + v);
                if (o >= lo && o < hi) atomicAnd(bits_cur + (g >> 5), ~(1u << (g & 31)));  // consumed
                val = ld_cg(a.f + g);
            }
            const int stop = min(hi, __shfl_sync(FULL, oend, 31));
            push_edges<MULTI, T>(a, r, beg, o, val, vw, x, stop, L);
            x = stop;
            i += 32;
        }
        // the local worklist after each chunk, while its vertices are near the sweep
        drain_local<MULTI, T>(a, r, red, L);
    }
    stage_flush(L.next_pull);
    stage_flush(L.next_push);
}

// ---------------------------------------------------------------------------
// Persistent fixpoint kernel (Algorithm 3's while-loop on the device).
template <bool MULTI, typename T>
__global__ void __launch_bounds__(THREADS, EG_FIXPOINT_MIN_BLOCKS) k_fixpoint(Args<T> a) {
    __shared__ T red_all[WARPS][32];
    __shared__ int stack_all[WARPS][LOCAL_CAP];
    __shared__ int stage_all[WARPS][4][STAGE];
    const int wid = threadIdx.x >> 5;
    T *red = red_all[wid];
    Local<T> L;
    L.stack = stack_all[wid];
    L.next_pull.item = stage_all[wid][0];
    L.next_pull.work = stage_all[wid][1];
    L.next_push.item = stage_all[wid][2];
    L.next_push.work = stage_all[wid][3];
    L.top = 0;
    L.on = false;
    L.relax = L.lifts = L.pushes = 0;
    Ctrl *c = a.ctrl;
    unsigned gen = ld_cg(&c->bar_gen);
    if (blockIdx.x == 0 && threadIdx.x == 0) c->stop_flag = 0;
    long long r_next = 0;
    for (int r = (int)a.r0;; ++r) {
        if (a.max_rounds > 0 && r >= a.max_rounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0 && !a.slice) atomicExch(&c->status, DEV_BUDGET);
            r_next = r;
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->pull_ctr[(r + 2) % 3] = 0;
            c->push_ctr[(r + 2) % 3] = 0;
            // round r + 1's take counters (round r's were cleared one round
            // earlier, or by the launch's reset of the control block)
            c->pull_take[(r + 1) % 3] = 0;
            c->push_take[(r + 1) % 3] = 0;
        }
        const unsigned long long pc = ld_cg(&c->pull_ctr[r % 3]);
        if ((pc & 0xffffffffu) != 0) {
            Stager out{L.next_push.item, L.next_push.work, 0, &c->push_ctr[r % 3], a.push_items[r & 1],
                       a.push_offs[r & 1]};
            pull_phase<MULTI, T>(a, r, red, out);
            stage_flush(out);
            if (!grid_barrier(c, gridDim.x, gen, a.wait_ns)) break;
        }
        const unsigned long long qc = ld_cg(&c->push_ctr[r % 3]);
        push_phase<MULTI, T>(a, r, red, L);
        if (a.doorbell && blockIdx.x == 0 && threadIdx.x == 0 && *a.doorbell) c->stop_flag = 1;
        if (!grid_barrier(c, gridDim.x, gen, a.wait_ns)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->rounds += 1;
            c->lifts += pc & 0xffffffffu;
            c->pushes += qc & 0xffffffffu;
            c->relax += (pc >> 32) + (qc >> 32);
        }
        const unsigned long long np = ld_cg(&c->pull_ctr[(r + 1) % 3]);
        const unsigned long long nq = ld_cg(&c->push_ctr[(r + 1) % 3]);
        if (blockIdx.x == 0 && threadIdx.x == 0) c->enqueues += (np & 0xffffffffu) + (nq & 0xffffffffu);
        r_next = r + 1;
        if ((np & 0xffffffffu) == 0 && (nq & 0xffffffffu) == 0) break;
        if (a.doorbell && ld_cg(&c->stop_flag)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) c->r_next = r_next;
    if (lane_id() == 0 && (L.relax | L.lifts | L.pushes)) {
        atomicAdd(&c->relax, L.relax);
        atomicAdd(&c->lifts, L.lifts);
        atomicAdd(&c->pushes, L.pushes);
    }
}

// ---------------------------------------------------------------------------
// Cycle jumps (accelerated lifting).  A cycle c of the arena whose weight
// under the view is negative cannot be followed for ever by the least
// fixpoint: each lap would need d more credit.  So some player-0 vertex of c
// leaves it, at a credit at or above its best other option.  With credits f
// at or below the least fixpoint and, for each player-0 vertex u of c,
// alt(u) = min over u's other edges of f(x) (-) w, the greatest solution of
//   x(v) = x(next) (-) w             (player 1)
//   x(v) = min(x(next) (-) w, alt(v)) (player 0)
// around c bounds the least fixpoint from below on c.  Raising f to x is
// therefore sound, and it ends in one step a climb that the lifting would
// take one lap per deficit d for.  The cycles tried are those of the
// current choices (each vertex's best edge under f), which are the cycles
// such climbs run on.

constexpr int KICK_LEN = 32;      // longest choice cycle jumped
constexpr int KICK_MAXDEG = 64;   // vertices of larger out-degree have no choice

// The current choice of vertex x (the edge of its lift's min or max under f)
// and, for a player-0 vertex, the best of its other edges; false if x has
// none (at TOP, frozen, or of out-degree above KICK_MAXDEG).
template <typename T>
__device__ __forceinline__ bool choice_of(const Args<T> &a, int x, int &edge, T &alt) {
    const DevArena &A = a.A;
    const int b = __ldg(A.row_ptr + x), e1 = __ldg(A.row_ptr + x + 1);
    if (e1 - b > KICK_MAXDEG || ld_cg(a.f + x) == Cred<T>::TOP) return false;
    if (a.frozen && ((__ldg(a.frozen + (x >> 5)) >> (x & 31)) & 1u)) return false;
    const bool p1 = ((__ldg(A.owner_bits + (x >> 5)) >> (x & 31)) & 1u) ^ a.inv;
    T best = p1 ? T(0) : Cred<T>::TOP, second = Cred<T>::TOP;
    int be = -1;
    for (int e = b; e < e1; ++e) {
        const T t = ominus<T>(ld_cg(a.f + __ldg(A.col + e)), wmap(__ldg(A.w + e), a.W), a.W.C);
        if (p1) {
            if (be < 0 || t > best) {
                best = t;
                be = e;
            }
        } else if (be < 0 || t < best) {
            second = best;
            best = t;
            be = e;
        } else if (t < second) {
            second = t;
        }
    }
    edge = be;
    alt = second;
    return be >= 0;
}

// One thread per entry of round r's pull and push lists: the walk along the
// current choices from the entry, computed as it goes; if it returns to the
// entry within KICK_LEN edges and the cycle's weight is negative, the cycle
// is claimed for this epoch at its smallest vertex (one jump per cycle),
// raised to its bound, and the vertices that rose join round r's push list.
// A climbing cycle always has a vertex in the lists, so scanning them finds
// the climbs at a cost that follows the frontier, not n.
template <typename T>
__global__ void k_jump(Args<T> a, int r, unsigned epoch, unsigned *claim, unsigned long long *jumped) {
    const DevArena &A = a.A;
    const int np = (int)(ld_cg(&a.ctrl->pull_ctr[r % 3]) & 0xffffffffu);
    const int nq = (int)(ld_cg(&a.ctrl->push_ctr[r % 3]) & 0xffffffffu);
    const int *pull = a.pull_items[r & 1], *push = a.push_items[r & 1];
    unsigned long long mine = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np + nq; i += gridDim.x * blockDim.x) {
        const int v = (i < np ? ld_cg(pull + i) : ld_cg(push + (i - np))) & 0x7fffffff;
        int cyc[KICK_LEN];
        T alts[KICK_LEN];
        int len = 0, x = v, lo = v;
        long long wsum = 0;
        bool closed = false;
        while (len < KICK_LEN) {
            int e;
            T al;
            if (!choice_of<T>(a, x, e, al)) break;
            cyc[len] = e;
            alts[len] = al;
            ++len;
            wsum += wmap(__ldg(A.w + e), a.W);
            x = __ldg(A.col + e);
            if (x == v) {
                closed = true;
                break;
            }
            lo = min(lo, x);
        }
        if (!closed || wsum >= 0) continue;
        if (atomicExch(claim + lo, epoch) == epoch) continue;  // jumped from another entry
        // greatest solution around the cycle, from TOP: two backward laps
        T xv[KICK_LEN];
        for (int k = 0; k < len; ++k) xv[k] = Cred<T>::TOP;
        for (int lap = 0; lap < 2; ++lap) {
            for (int k = len - 1; k >= 0; --k) {
                const int cv = k == 0 ? v : __ldg(A.col + cyc[k - 1]);
                T val = ominus<T>(xv[k + 1 == len ? 0 : k + 1], wmap(__ldg(A.w + cyc[k]), a.W), a.W.C);
                const bool p1 = ((__ldg(A.owner_bits + (cv >> 5)) >> (cv & 31)) & 1u) ^ a.inv;
                if (!p1) val = min(val, alts[k]);
                xv[k] = val;
            }
        }
        for (int k = 0; k < len; ++k) {
            const int cv = k == 0 ? v : __ldg(A.col + cyc[k - 1]);
            if (!(xv[k] > ld_cg(a.f + cv))) continue;
            if (!(xv[k] > atomicMax(a.f + cv, xv[k]))) continue;
            ++mine;
            const int work = __ldg(A.rrow_ptr + cv + 1) - __ldg(A.rrow_ptr + cv);
            const unsigned bit = 1u << (cv & 31);
            if (work > 0 && !(atomicOr(a.bits_push[r & 1] + (cv >> 5), bit) & bit)) {
                const unsigned long long base =
                    atomicAdd(&a.ctrl->push_ctr[r % 3], ((unsigned long long)(unsigned)work << 32) | 1ull);
                const unsigned idx = (unsigned)(base & 0xffffffffu);
                a.push_items[r & 1][idx] = cv;
                a.push_offs[r & 1][idx] = (int)(base >> 32);
            }
        }
    }
    for (int d = 16; d; d >>= 1) mine += __shfl_down_sync(FULL, mine, d);
    if (lane_id() == 0 && mine) atomicAdd(jumped, mine);
}

// ---------------------------------------------------------------------------
// Host side

// A persistent fixpoint kernel waits at grid barriers for all its blocks.
// Two of them on one device at once can each end up partly resident, the
// resident blocks of each waiting for blocks that cannot start until the
// other grid's blocks leave; the barrier's wait limit then ends both with
// EG_ERR_TIMEOUT.  So within the process the library runs one persistent
// solve per device at a time: every route that launches the fixpoint kernel
// holds its device's lock (recursive: routes nest) from before its first
// launch until its last synchronisation.
static std::recursive_mutex &persist_lock(int device) {
    static std::recursive_mutex locks[64];
    return locks[device >= 0 && device < 64 ? device : 0];
}

static int num_sms(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (device >= 0 && device < 64) cached[device] = sms;
    return sms;
}

eg_status compute_bound(eg_arena *ar, long long scale, long long shift, long long *C, long long *wmax,
                        cudaStream_t s) {
    if (scale == 1 && shift == 0 && ar->C_plain >= 0) {
        *C = ar->C_plain;
        *wmax = ar->wmax_plain;
        return EG_OK;
    }
    unsigned long long *d = nullptr, h[2] = {0, 0};
    EG_CUDA_TRY(cudaMallocAsync((void **)&d, 2 * sizeof(unsigned long long), s));
    EG_CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s));
    WeightView W{scale, shift, 0};
    int blocks = num_sms(ar->device) * 8;
    k_bound<<<blocks, 256, 0, s>>>(ar->d, W, d, d + 1);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaFreeAsync(d, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    *C = (long long)h[0];
    *wmax = (long long)h[1];
    if (scale == 1 && shift == 0) {
        ar->C_plain = *C;
        ar->wmax_plain = *wmax;
    }
    return EG_OK;
}

eg_status free_state(StateBuffers &sb) {
    if (sb.block) cudaFree(sb.block);
    sb = StateBuffers{};
    return EG_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Blocks of 256 threads for an O(n) pass over n credits.
static int wblocks_of(long long n, int sms) { return (int)std::min<long long>((n + 255) / 256, (long long)sms * 16); }

// Solve state for nf credits of the given width.
eg_status alloc_state(StateBuffers &sb, long long nf, int bits) {
    if (sb.bits == bits && sb.nf == nf) return EG_OK;
    free_state(sb);
    const size_t n = (size_t)nf, cs = bits / 8, words = (n + 31) / 32;
    size_t off = 0;
    size_t o_f = off; off = align_up(off + n * cs);
    size_t o_list[8];
    for (int k = 0; k < 8; ++k) { o_list[k] = off; off = align_up(off + n * 4); }
    size_t o_bits[5];
    for (int k = 0; k < 5; ++k) { o_bits[k] = off; off = align_up(off + words * 4); }
    size_t o_acc = off; off = align_up(off + n * cs);
    size_t o_done = off; off = align_up(off + n * 4);
    size_t o_ctrl = off; off = align_up(off + sizeof(Ctrl));
    char *blk = nullptr;
    EG_CUDA_TRY(cudaMalloc((void **)&blk, off));
    sb.block = blk;
    sb.bytes = off;
    sb.bits = bits;
    sb.nf = nf;
    sb.dirty = true;
    sb.d.f = blk + o_f;
    for (int k = 0; k < 2; ++k) {
        sb.d.pull_items[k] = (int *)(blk + o_list[4 * k + 0]);
        sb.d.pull_offs[k] = (int *)(blk + o_list[4 * k + 1]);
        sb.d.push_items[k] = (int *)(blk + o_list[4 * k + 2]);
        sb.d.push_offs[k] = (int *)(blk + o_list[4 * k + 3]);
        sb.d.bits_pull[k] = (unsigned *)(blk + o_bits[k]);
        sb.d.bits_push[k] = (unsigned *)(blk + o_bits[2 + k]);
    }
    sb.d.seed_bits = (unsigned *)(blk + o_bits[4]);
    sb.d.acc = blk + o_acc;
    sb.d.acc_done = (int *)(blk + o_done);
    sb.d.ctrl = (Ctrl *)(blk + o_ctrl);
    return EG_OK;
}

static eg_status ensure_state(eg_arena *ar, int bits) {
    return alloc_state(bits == 32 ? ar->st32 : ar->st64, ar->n, bits);
}

// Launch parameters shared by single and batched solves.
struct Launch {
    int local_windows, local_maxdeg, warm_start;
    long long seed_max_pairs, max_rounds;
    bool preseeded = false;  // seed_bits already holds proven TOP starts (kept; 2-cycle seeds are added)
    unsigned inv = 0;        // 1: owners swapped (dual game)
    int blocks_per_sm = 0;   // resident blocks per SM of the fixpoint kernel (0: as many as fit)
    unsigned long long wait_ns = BARRIER_LIMIT_NS;
    const unsigned *frozen = nullptr;  // vertices held at 0 (dual lifts of the certified trials)
    const int *level = nullptr;        // SCC-ordered solves: level of each vertex
    int cur_level = 0;                 //   and the level this launch solves (0 first)
    long long slice_rounds = 0;        // > 0: the launch stops after this many rounds, without error
    int chunk_edges = 0;               // edges per chunk of a long list (0: one chunk per warp)
    int sweeps = 0;                    // dense sweeps before the worklist rounds (not with levels)
    const int *tiles = nullptr;        // non-null: the tiles the O(n) passes visit (see Args)
    long long ntiles = 0;
};

// The arena's launch settings with the given warm start and round budget.
static Launch launch_of(const eg_arena *ar, int warm_start, long long max_rounds) {
    Launch L{ar->local_windows, ar->local_maxdeg, warm_start, ar->seed_max_pairs, max_rounds};
    L.blocks_per_sm = ar->blocks_per_sm;
    L.wait_ns = ar->wait_limit_ns;
    L.chunk_edges = ar->chunk_edges;
    L.sweeps = ar->sweeps;
    return L;
}

// Enqueues (warm start,) initialisation, the dense sweeps and the persistent
// fixpoint on stream s; ev_k (optional) is recorded right before the lifting
// kernels (the sweeps, or the fixpoint kernel when there are none).
template <bool MULTI, typename T>
static eg_status enqueue_solve(const DevArena &A, const WeightView &W, const InstTable &I, long long nf,
                               StateBuffers &sb, const Launch &L, int device, cudaStream_t s, cudaEvent_t ev_k,
                               Args<T> *keep = nullptr, int *grid_blocks = nullptr) {
    const int sms = num_sms(device);
    if (sb.dirty) {
        k_fill<T><<<sms * 4, 256, 0, s>>>((T *)sb.d.acc, nf, Cred<T>::TOP);
        EG_CUDA_TRY(cudaGetLastError());
        EG_CUDA_TRY(cudaMemsetAsync(sb.d.acc_done, 0, (size_t)nf * 4, s));
        for (int k = 0; k < 2; ++k) {
            EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits_pull[k], 0, ((size_t)nf + 31) / 32 * 4, s));
            EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits_push[k], 0, ((size_t)nf + 31) / 32 * 4, s));
        }
        sb.dirty = false;
    }
    EG_CUDA_TRY(cudaMemsetAsync(sb.d.ctrl, 0, sizeof(Ctrl), s));
    Args<T> a;
    a.A = A;
    a.W = W;
    a.I = I;
    a.nf = (int)nf;
    a.f = (T *)sb.d.f;
    for (int k = 0; k < 2; ++k) {
        a.pull_items[k] = sb.d.pull_items[k];
        a.pull_offs[k] = sb.d.pull_offs[k];
        a.push_items[k] = sb.d.push_items[k];
        a.push_offs[k] = sb.d.push_offs[k];
        a.bits_pull[k] = sb.d.bits_pull[k];
        a.bits_push[k] = sb.d.bits_push[k];
    }
    a.acc = (T *)sb.d.acc;
    a.acc_done = sb.d.acc_done;
    a.ctrl = sb.d.ctrl;
    a.max_rounds = L.slice_rounds > 0 ? L.slice_rounds : L.max_rounds;
    a.r0 = 0;
    a.slice = L.slice_rounds > 0 ? 1 : 0;
    a.doorbell = nullptr;
    a.local_windows = L.local_windows;
    a.local_maxdeg = L.local_maxdeg;
    a.chunk = L.chunk_edges;
    a.wait_ns = L.wait_ns;
    a.inv = L.inv;
    a.frozen = L.frozen;
    a.level = L.level;
    a.cur_level = L.cur_level;
    a.tiles = L.tiles;
    a.ntiles = L.ntiles;
    a.seed_bits = nullptr;
    const bool first = !L.level || L.cur_level == 0;  // an SCC-ordered solve seeds once, at level 0
    if (first && (L.warm_start || L.preseeded)) {
        if (!L.preseeded) EG_CUDA_TRY(cudaMemsetAsync(sb.d.seed_bits, 0, ((size_t)nf + 31) / 32 * 4, s));
        if (L.warm_start) {
            const int sblocks = (int)std::min<long long>((nf + 7) / 8, (long long)sms * 32);
            k_seed<MULTI, T><<<sblocks, 256, 0, s>>>(a, L.seed_max_pairs, sb.d.seed_bits, &sb.d.ctrl->seeded, 0,
                                                     (int)nf);
            EG_CUDA_TRY(cudaGetLastError());
        }
        a.seed_bits = sb.d.seed_bits;
    }
    const int init_blocks = (int)std::min<long long>((nf + THREADS - 1) / THREADS, (long long)sms * 16);
    if (L.level) {
        if (first)
            k_level_start<T><<<init_blocks, THREADS, 0, s>>>(a.f, (int)nf, a.seed_bits);
        k_init_level<T><<<init_blocks, THREADS, 0, s>>>(a, L.cur_level);
    } else {
        k_init<MULTI, T><<<init_blocks, THREADS, 0, s>>>(a, 0, (int)nf, 0, 0, L.sweeps > 0 ? 0 : 1);
        EG_CUDA_TRY(cudaGetLastError());
        if (ev_k && L.sweeps > 0) EG_CUDA_TRY(cudaEventRecord(ev_k, s));  // the lifting starts with the sweeps
        if (L.sweeps > 0) {
            static int sweep_per_sm[64] = {0};  // resident sweep blocks per SM, per device
            int sp = device >= 0 && device < 64 ? sweep_per_sm[device] : 0;
            if (sp < 1) {
                EG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sp, k_sweep<MULTI, T>, THREADS, 0));
                sp = std::max(sp, 1);
                if (device >= 0 && device < 64) sweep_per_sm[device] = sp;
            }
            // one resident wave: the grid moves through the credits together
            const int sw_blocks = (int)std::min<long long>((nf + THREADS - 1) / THREADS, (long long)sms * sp);
            for (int k = 0; k < L.sweeps; ++k)
                k_sweep<MULTI, T><<<sw_blocks, THREADS, 0, s>>>(a, k == L.sweeps - 1 ? 1 : 0);
        }
    }
    EG_CUDA_TRY(cudaGetLastError());

    static int per_sm_cache[64] = {0};  // resident blocks per SM, per device
    int per_sm = device >= 0 && device < 64 ? per_sm_cache[device] : 0;
    if (per_sm < 1) {
        EG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fixpoint<MULTI, T>, THREADS, 0));
        if (per_sm < 1) {
            set_error("fixpoint kernel cannot be resident");
            return EG_ERR_CUDA;
        }
        if (device >= 0 && device < 64) per_sm_cache[device] = per_sm;
    }
    if (L.blocks_per_sm > 0) per_sm = std::min(per_sm, L.blocks_per_sm);
    dim3 grid(sms * per_sm), block(THREADS);
    void *args[] = {&a};
    if (ev_k && (L.sweeps == 0 || L.level)) EG_CUDA_TRY(cudaEventRecord(ev_k, s));
    EG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_fixpoint<MULTI, T>, grid, block, args, 0, s));
    if (keep) *keep = a;  // for the launches that resume it
    if (grid_blocks) *grid_blocks = (int)grid.x;
    return EG_OK;
}

template <typename T>
static eg_status launch_solve(eg_arena *ar, StateBuffers &sb, const WeightView &W, cudaStream_t s, const Launch &L) {
    EG_CUDA_TRY(cudaEventRecord(ar->ev0, s));
    InstTable none{1, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
    eg_status rc = enqueue_solve<false, T>(ar->d, W, none, ar->n, sb, L, ar->device, s, ar->evk);
    if (rc != EG_OK) return rc;
    EG_CUDA_TRY(cudaEventRecord(ar->ev1, s));
    return EG_OK;
}

__global__ void k_widen(const int *in, long long *out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int v = in[i];
        out[i] = v == Cred<int>::TOP ? Cred<long long>::TOP : (long long)v;
    }
}

// ---------------------------------------------------------------------------
// Certified trial caps.
//
// The least fixpoint with a cap B below C is pointwise at or above the one
// with cap C (the capped (-) only reaches TOP sooner), so a vertex finite
// under cap B is won by player 0.  The same holds in the dual game: weights
// -(K w' + 1) for some K >= 1, owners swapped, so that player 1 is the
// energy player.  A vertex finite there is won by player 1 in the dual, i.e.
// player 1 has a positional strategy under which every cycle c of the play
// has K w'(c) + |c| <= 0, hence w'(c) < 0: player 1 wins the game itself
// from it (Lemma "EGcycles"), so its least-EPM value is TOP.  Proven player-1
// vertices start the next lift of the game at TOP, proven player-0 vertices
// start the next lift of the dual at TOP; both starts stay below the least
// fixpoint they lift towards.  When, after a capped lift of the game, every
// vertex is finite or proven lost, every credit player 0 wins is at most its
// capped value, so at most B; a cap at or above the largest finite credit
// gives the same least fixpoint as C (Sec. 3.1 needs M_G only as an upper
// bound on finite credits), so the capped result is exact.
//
// A larger K proves more (a cycle of length L and weight -s needs K >= L/s),
// but the dual credits grow with K and so do the climbs that reach them:
// the trials start at a small K (EG_OPT_DUAL_K, 4) and a small B and grow
// both; from the second trial on the proven losses are frozen in the dual,
// so its lift touches only the vertices still undecided.

// OR of the finite credits into a bitmap (one warp per bitmap word).  With
// an instance table that has an `active` array (batched solves), only the
// credits of active instances count: the others were not computed by the
// launch just run.
template <typename T>
__global__ void k_mark_finite(const T *f, int n, unsigned *bits, InstTable I, const int *tiles, long long ntiles) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const long long nt = tile_count(tiles, ntiles, 0, n);
    for (long long t = gw; t < nt; t += nw) {
        const int base = tile_base(tiles, t, 0);
        const int g = base + lane;
        bool fin = g < n && f[g] != Cred<T>::TOP;
        if (fin && I.active) fin = __ldg(I.active + inst_of(I, g)) != 0;
        const unsigned word = __ballot_sync(FULL, fin);
        if (lane == 0 && word) bits[base >> 5] |= word;
    }
}

// dst |= src over `words` bitmap words.
__global__ void k_or_bits(unsigned *dst, const unsigned *src, int words) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) dst[i] |= src[i];
}

// count[0] += credits at TOP that no proof puts in W1; count[1] += proven W1.
template <typename T>
__global__ void k_count_undecided(const T *f, const unsigned *w1, int n, unsigned long long *count) {
    unsigned long long und = 0, proven = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const bool p = (w1[g >> 5] >> (g & 31)) & 1u;
        proven += p;
        und += f[g] == Cred<T>::TOP && !p;
    }
    for (int d = 16; d; d >>= 1) {
        und += __shfl_down_sync(FULL, und, d);
        proven += __shfl_down_sync(FULL, proven, d);
    }
    if (lane_id() == 0) {
        if (und) atomicAdd(count, und);
        if (proven) atomicAdd(count + 1, proven);
    }
}

// Per-instance count of credits at TOP that no proof puts in W1 (a warp
// whose credits all belong to one instance adds them with one atomic).
template <typename T>
__global__ void k_count_undecided_inst(const T *f, const unsigned *w1, InstTable I, int nf,
                                       unsigned long long *count, const int *tiles, long long ntiles) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const long long nt = tile_count(tiles, ntiles, 0, nf);
    for (long long t = gw; t < nt; t += nw) {
        const int g = tile_base(tiles, t, 0) + lane;
        int i = -1;
        unsigned long long und = 0;
        if (g < nf) {
            i = inst_of(I, g);
            und = f[g] == Cred<T>::TOP && !((w1[g >> 5] >> (g & 31)) & 1u);
        }
        const int i0 = __shfl_sync(FULL, i, 0);
        if (__all_sync(FULL, i == i0)) {
            for (int d = 16; d; d >>= 1) und += __shfl_down_sync(FULL, und, d);
            if (lane == 0 && und) atomicAdd(count + i0, und);
        } else if (und) {
            atomicAdd(count + i, und);
        }
    }
}

// Marks the instance of every entry of the pull and push lists of round r
// (list counter `slot`) of a batched solve.
__global__ void k_busy_plan(const Ctrl *c, int slot, const int *pull_items, const int *push_items, InstTable I,
                            int *busy) {
    const int np = (int)(ld_cg(&c->pull_ctr[slot]) & 0xffffffffu);
    const int nq = (int)(ld_cg(&c->push_ctr[slot]) & 0xffffffffu);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np + nq; i += gridDim.x * blockDim.x) {
        const int g = (i < np ? ld_cg(pull_items + i) : ld_cg(push_items + (i - np))) & 0x7fffffff;
        busy[inst_of(I, g)] = 1;
    }
}

// Counters summed over the fixpoint launches of one solve, with one record
// per launch (its kind, cap, rounds, relaxations and kernel time).
struct PhaseRec {
    int kind;
    long long cap, rounds, relax;
    double kms;
};

struct Totals {
    long long rounds = 0, lifts = 0, pushes = 0, relax = 0, enqueues = 0, seeded = 0, jumps = 0;
    double ms = 0, kms = 0;
    int trials = 0;
    std::vector<PhaseRec> phases;
};

// Adds the counters of the launch whose control block was just read back
// into `hc`; ms and kms are its device times (whole solve, fixpoint kernel).
static void add_launch(Totals &t, const Ctrl *hc, double ms, double kms, int kind, long long cap) {
    t.rounds += (long long)hc->rounds;
    t.lifts += (long long)hc->lifts;
    t.pushes += (long long)hc->pushes;
    t.relax += (long long)hc->relax;
    t.enqueues += (long long)hc->enqueues;
    t.seeded = std::max(t.seeded, (long long)hc->seeded);
    t.ms += ms;
    t.kms += kms;
    t.phases.push_back(PhaseRec{kind, cap, (long long)hc->rounds, (long long)hc->relax, kms});
}

static void add_totals(Totals &t, const eg_arena *ar, int kind, long long cap) {
    float ms = 0.f, kms = 0.f;
    cudaEventElapsedTime(&ms, ar->ev0, ar->ev1);
    cudaEventElapsedTime(&kms, ar->evk, ar->ev1);
    add_launch(t, (const Ctrl *)ar->host_ctrl, ms, kms, kind, cap);
}

static void fill_stats(eg_stats *st, const Totals &t, long long C, long long seeded, int bits, eg_status result) {
    st->C = C;
    st->seeded = seeded;
    st->credit_bits = bits;
    st->status = result;
    st->rounds = t.rounds;
    st->lifts = t.lifts;
    st->pushes = t.pushes;
    st->relaxations = t.relax;
    st->enqueues = t.enqueues;
    st->ms = t.ms;
    st->fixpoint_ms = t.kms;
    st->cycle_jumps = t.jumps;
    st->phases = (int32_t)std::min<size_t>(t.phases.size(), EG_MAX_PHASES);
    st->trials = t.trials;
    for (int k = 0; k < EG_MAX_PHASES; ++k) {
        const bool have = k < st->phases;
        st->phase_kind[k] = have ? t.phases[k].kind : 0;
        st->phase_cap[k] = have ? t.phases[k].cap : 0;
        st->phase_rounds[k] = have ? t.phases[k].rounds : 0;
        st->phase_relaxations[k] = have ? t.phases[k].relax : 0;
        st->phase_ms[k] = have ? t.phases[k].kms : 0.0;
    }
}

// Where one single-game solve keeps its working memory: the game's state (of
// the solve's credit width), the int64 state of the dual lifts, and the
// certified trials' bitmaps of proven player-0 and player-1 vertices with two
// counters.  eg_solve_credit takes them from the arena and allocates them on
// first use; eg_solve_credit_noalloc lays them over its fixed device array,
// where the two states share their lists, bitmaps and scratch (so every
// launch there resets that scratch first).
struct SolveMem {
    StateBuffers *sb = nullptr;
    StateBuffers *sd = nullptr;
    unsigned *cert_w0 = nullptr, *cert_w1 = nullptr;
    unsigned long long *aux = nullptr;
    bool fixed = false;     // laid over the allocation-free array
    bool in_place = false;  // sb's credit array is the caller's output buffer
    long long attempt_only = 0;  // > 0: only a first attempt of this many rounds (EG_ERR_BUDGET if unfinished)
    unsigned *kick_claim = nullptr;  // cycle jumps: the epoch each vertex's cycle was last jumped in,
    unsigned *kick_epoch = nullptr;  //   the epoch counter of that array (host),
    unsigned long long *kick_jumps = nullptr;  //   and the count of vertices raised
};

// Next epoch of a claim array; on wrap-around the array is cleared (0 is
// never an epoch).
static eg_status next_epoch(unsigned *claim, unsigned *epoch, long long n, cudaStream_t s, unsigned &out) {
    if (++*epoch == 0) {
        EG_CUDA_TRY(cudaMemsetAsync(claim, 0, (size_t)n * 4, s));
        *epoch = 1;
    }
    out = *epoch;
    return EG_OK;
}

// The scratch of the cycle jumps of an allocating solve (allocated and
// cleared on first use): a claim epoch per vertex and a counter.
static eg_status kick_memory(eg_arena *ar, SolveMem &m) {
    if (m.kick_claim) return EG_OK;
    const size_t o_cnt = align_up((size_t)ar->n * 4);
    if (!ar->kick_block) {
        EG_CUDA_TRY(cudaMalloc(&ar->kick_block, o_cnt + 256));
        EG_CUDA_TRY(cudaMemset(ar->kick_block, 0, o_cnt + 256));
        ar->kick_epoch = 0;
    }
    m.kick_claim = (unsigned *)ar->kick_block;
    m.kick_epoch = &ar->kick_epoch;
    m.kick_jumps = (unsigned long long *)((char *)ar->kick_block + o_cnt);
    return EG_OK;
}

// The dual state and the trial bitmaps of an allocating solve.
static eg_status cert_memory(eg_arena *ar, SolveMem &m) {
    if (m.fixed) return EG_OK;
    // the dual lifts get their own state: the capped fixpoint of the game
    // stays in m.sb while the dual runs
    eg_status rc = alloc_state(ar->st_dual, ar->n, 64);
    if (rc != EG_OK) return rc;
    m.sd = &ar->st_dual;
    if (!ar->cert_block) {
        const size_t words = ((size_t)ar->n + 31) / 32, bm = align_up(words * 4);
        char *blk = nullptr;
        EG_CUDA_TRY(cudaMalloc((void **)&blk, 256 + 2 * bm));
        ar->cert_block = blk;
        ar->aux = (unsigned long long *)blk;
        ar->cert_w0 = (unsigned *)(blk + 256);
        ar->cert_w1 = (unsigned *)(blk + 256 + bm);
    }
    m.cert_w0 = ar->cert_w0;
    m.cert_w1 = ar->cert_w1;
    m.aux = ar->aux;
    return EG_OK;
}

// One solve run to its end on s; adds its counters and returns its device
// status.  With cycle jumps on (EG_OPT_KICK_ROUNDS > 0, not for the levels
// of an SCC-ordered solve), the fixpoint runs in slices of that many rounds
// and the choice cycles are jumped between slices; a slice resumes at the
// round the last one stopped at, with its lists.
template <typename T>
static eg_status run_phase(eg_arena *ar, SolveMem &m, StateBuffers &sb, const WeightView &W, const Launch &L,
                           cudaStream_t s, Totals &t, int kind, int &dev) {
    if (m.fixed) sb.dirty = true;  // the scratch is shared with the other state
    const long long R = ar->kick_rounds;
    eg_status rc = EG_OK;
    if (R <= 0 || L.level) {
        rc = launch_solve<T>(ar, sb, W, s, L);
        if (rc != EG_OK) return rc;
        EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        add_totals(t, ar, kind, W.C);
        dev = ((const Ctrl *)ar->host_ctrl)->status;
        if (dev != DEV_OK) sb.dirty = true;
        return EG_OK;
    }
    if ((rc = kick_memory(ar, m)) != EG_OK) return rc;
    const int sms = num_sms(ar->device);
    EG_CUDA_TRY(cudaMemsetAsync(m.kick_jumps, 0, sizeof(unsigned long long), s));
    EG_CUDA_TRY(cudaEventRecord(ar->ev0, s));
    Launch Ls = L;
    Ls.slice_rounds = L.max_rounds > 0 ? std::min(R, L.max_rounds) : R;
    Args<T> a;
    int blocks = 0;
    const InstTable none{1, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
    rc = enqueue_solve<false, T>(ar->d, W, none, ar->n, sb, Ls, ar->device, s, ar->evk, &a, &blocks);
    if (rc != EG_OK) return rc;
    const Ctrl *hc = (const Ctrl *)ar->host_ctrl;
    bool budget = false;
    for (;;) {
        EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        if (hc->status != DEV_OK) break;
        const long long r = hc->r_next;
        const long long entries = (long long)(hc->pull_ctr[r % 3] & 0xffffffffu) + (hc->push_ctr[r % 3] & 0xffffffffu);
        if (entries == 0) break;
        if (L.max_rounds > 0 && r >= L.max_rounds) {
            budget = true;
            break;
        }
        unsigned epoch = 0;
        if ((rc = next_epoch(m.kick_claim, m.kick_epoch, ar->n, s, epoch)) != EG_OK) return rc;
        const int jb = (int)std::min<long long>((entries + 255) / 256, (long long)sms * 8);
        k_jump<T><<<jb, 256, 0, s>>>(a, (int)r, epoch, m.kick_claim, m.kick_jumps);
        EG_CUDA_TRY(cudaGetLastError());
        a.r0 = r;
        a.max_rounds = L.max_rounds > 0 ? std::min(r + R, L.max_rounds) : r + R;
        void *args[] = {&a};
        EG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_fixpoint<false, T>, dim3(blocks), dim3(THREADS), args,
                                                0, s));
    }
    EG_CUDA_TRY(cudaEventRecord(ar->ev1, s));
    unsigned long long jumps = 0;
    EG_CUDA_TRY(cudaMemcpyAsync(&jumps, m.kick_jumps, sizeof(jumps), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    add_totals(t, ar, kind, W.C);
    t.jumps += (long long)jumps;
    dev = budget ? DEV_BUDGET : hc->status;
    if (dev != DEV_OK) sb.dirty = true;
    return EG_OK;
}

constexpr int CERT_TRIALS = 6;

// Trials k = 0..5 with B = cap_certify * max|w'| * 4^k and K = dual_k * 8^k
// (at most n + 1).  A trial first lifts the game with cap B from the proven
// player-1 vertices at TOP; its finite vertices are proven player-0 wins.
// If every vertex is then finite or proven lost, that capped fixpoint is
// the least one.  Otherwise the dual is lifted with the proven player-0
// vertices at TOP and the proven player-1 vertices frozen at 0 (sinks of the
// dual: a vertex that is finite there is lost by player 0, because player 1
// either keeps the play on negative cycles or reaches a vertex already
// proven lost), and the count is taken again over the same capped fixpoint.
// exact: m.sb holds the least fixpoint.  seeded: m.cert_w1 holds proven TOP
// starts for a final solve with cap C.
template <typename T>
static eg_status certify(eg_arena *ar, SolveMem &m, long long scale, long long shift, long long C, long long wmax,
                         cudaStream_t s, long long max_rounds, Totals &t, int &dev, bool &exact, bool &seeded,
                         long long &nproven) {
    exact = seeded = false;
    dev = DEV_OK;
    if (ar->cap_certify <= 0 || !ar->warm_start) return EG_OK;
    constexpr long long LIM = 1LL << 61;
    const long long n = ar->n;
    // |K w'| and the dual's intermediate K * scale * w stay below 2^61
    const long long inner = (scale < 0 ? -scale : scale) * std::max(1LL, ar->wmax_plain) +
                            (shift < 0 ? -shift : shift) + 1;
    if (wmax > LIM / 4 / ar->cap_certify) return EG_OK;
    long long B = (long long)ar->cap_certify * std::max(1LL, wmax);
    if (B >= C) return EG_OK;
    eg_status rc = cert_memory(ar, m);
    if (rc != EG_OK) return rc;
    StateBuffers &sb = *m.sb, &sd = *m.sd;
    const size_t words = ((size_t)n + 31) / 32;
    EG_CUDA_TRY(cudaMemsetAsync(m.cert_w0, 0, words * 4, s));
    EG_CUDA_TRY(cudaMemsetAsync(m.cert_w1, 0, words * 4, s));
    const int sms = num_sms(ar->device);
    const int wblocks = (int)std::min<long long>((n + 255) / 256, (long long)sms * 16);
    const InstTable all{};
    unsigned long long *h = (unsigned long long *)ar->host_ctrl;
    // A lift whose cap and weights fit int32 runs in int32 state: half the
    // bytes per credit (a 16M-vertex credit array then fits in L2).  Not in
    // the allocation-free array, which has one layout.
    auto fits32 = [](long long cap, long long wm) { return cap + wm <= 0x7fffffffLL - 1; };
    // h[0] = credits of the capped fixpoint (f, of width w) at TOP without a
    // proof of loss, h[1] = proven losses
    auto count = [&](const void *f, int w) -> eg_status {
        EG_CUDA_TRY(cudaMemsetAsync(m.aux, 0, 2 * sizeof(unsigned long long), s));
        if (w == 32) k_count_undecided<int><<<wblocks, 256, 0, s>>>((const int *)f, m.cert_w1, (int)n, m.aux);
        else k_count_undecided<long long><<<wblocks, 256, 0, s>>>((const long long *)f, m.cert_w1, (int)n, m.aux);
        EG_CUDA_TRY(cudaGetLastError());
        EG_CUDA_TRY(cudaMemcpyAsync(h, m.aux, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        nproven = (long long)h[1];
        return EG_OK;
    };
    long long K = std::min((long long)ar->dual_k, n + 1);
    for (int k = 0; k < CERT_TRIALS && B < C; ++k) {
        if (K > LIM / inner || B > LIM / (K + 1)) break;
        t.trials = k + 1;
        // the game with cap B: proven player-1 vertices start at TOP
        const bool narrow = sizeof(T) == 8 && !m.fixed && fits32(B, wmax);
        if (narrow && (rc = ensure_state(ar, 32)) != EG_OK) return rc;
        StateBuffers &sc = narrow ? ar->st32 : sb;  // the capped lift's state
        const int cw = narrow ? 32 : (int)sizeof(T) * 8;
        EG_CUDA_TRY(cudaMemcpyAsync(sc.d.seed_bits, m.cert_w1, words * 4, cudaMemcpyDeviceToDevice, s));
        Launch Lp = launch_of(ar, 1, max_rounds);
        Lp.preseeded = true;
        rc = narrow ? run_phase<int>(ar, m, sc, WeightView{scale, shift, B}, Lp, s, t, EG_PHASE_CAPPED, dev)
                    : run_phase<T>(ar, m, sc, WeightView{scale, shift, B}, Lp, s, t, EG_PHASE_CAPPED, dev);
        if (rc != EG_OK || dev != DEV_OK) return rc;
        seeded = true;
        // the warm start's own finds are proven losses too
        k_or_bits<<<(int)std::min<size_t>((words + 255) / 256, 1024), 256, 0, s>>>(m.cert_w1, sc.d.seed_bits,
                                                                                   (int)words);
        if (cw == 32) k_mark_finite<int><<<wblocks, 256, 0, s>>>((const int *)sc.d.f, (int)n, m.cert_w0, all, nullptr, 0);
        else k_mark_finite<long long><<<wblocks, 256, 0, s>>>((const long long *)sc.d.f, (int)n, m.cert_w0, all, nullptr, 0);
        EG_CUDA_TRY(cudaGetLastError());
        // an exact capped fixpoint computed in int32 goes to the solve's own
        // state, where the output and an in-place caller find it
        auto finish = [&]() -> eg_status {
            exact = true;
            if (narrow) {
                k_widen<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(
                    (const int *)sc.d.f, (long long *)sb.d.f, (int)n);
                EG_CUDA_TRY(cudaGetLastError());
            }
            return EG_OK;
        };
        if ((rc = count(sc.d.f, cw)) != EG_OK) return rc;
        if (h[0] == 0) return finish();
        // the dual: proven player-0 vertices start at TOP, proven player-1
        // vertices are held at 0
        const bool narrow_d = !m.fixed && fits32((K + 1) * B, K * wmax + 1);
        if (narrow_d && (rc = alloc_state(ar->st_dual32, ar->n, 32)) != EG_OK) return rc;
        StateBuffers &sdd = narrow_d ? ar->st_dual32 : sd;
        EG_CUDA_TRY(cudaMemcpyAsync(sdd.d.seed_bits, m.cert_w0, words * 4, cudaMemcpyDeviceToDevice, s));
        Launch Ld = launch_of(ar, 1, max_rounds);
        Ld.inv = 1;
        Ld.preseeded = true;
        Ld.frozen = m.cert_w1;
        const WeightView Wd{-K * scale, 1 - K * shift, (K + 1) * B};
        rc = narrow_d ? run_phase<int>(ar, m, sdd, Wd, Ld, s, t, EG_PHASE_DUAL, dev)
                      : run_phase<long long>(ar, m, sdd, Wd, Ld, s, t, EG_PHASE_DUAL, dev);
        if (rc != EG_OK || dev != DEV_OK) return rc;
        if (narrow_d) k_mark_finite<int><<<wblocks, 256, 0, s>>>((const int *)sdd.d.f, (int)n, m.cert_w1, all, nullptr, 0);
        else k_mark_finite<long long><<<wblocks, 256, 0, s>>>((const long long *)sdd.d.f, (int)n, m.cert_w1, all, nullptr, 0);
        EG_CUDA_TRY(cudaGetLastError());
        if ((rc = count(sc.d.f, cw)) != EG_OK) return rc;
        if (h[0] == 0) return finish();
        if (B > LIM / 4) break;
        B *= 4;
        K = std::min(K * 8, n + 1);
    }
    return EG_OK;
}

// Queues the copy of the credits of sb to out (host or device): same width,
// or widened to int64 with TOP mapped when credit_bits == 0.
static eg_status enqueue_output(eg_arena *ar, StateBuffers &sb, int bits, int credit_bits, void *out,
                                cudaStream_t s) {
    const int out_bits = credit_bits == 0 ? 64 : bits;
    cudaPointerAttributes attr{};
    const bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess &&
                         (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    void *src = sb.d.f;
    void *tmp = nullptr;
    if (out_bits != bits) {
        EG_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)ar->n * 8, s));
        const int wb = std::min((ar->n + 255) / 256, 4096);
        k_widen<<<wb, 256, 0, s>>>((const int *)sb.d.f, (long long *)tmp, ar->n);
        EG_CUDA_TRY(cudaGetLastError());
        src = tmp;
    }
    EG_CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)ar->n * (out_bits / 8),
                                dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (tmp) EG_CUDA_TRY(cudaFreeAsync(tmp, s));
    return EG_OK;
}

// The route of one single-game solve, in the memory m gives it: a first
// lift with cap C under a short round budget; if it does not finish, the
// certified trials; if they decide nothing, a final lift with cap C from
// their proven TOP starts.  bits is the width of m.sb; unless m.in_place,
// the credits are then copied to out (widened when credit_bits is 0).
static eg_status solve_route(eg_arena *ar, SolveMem &m, int bits, int credit_bits, long long scale, long long shift,
                             long long C, long long wmax, void *out, eg_stats *st, cudaStream_t s,
                             long long max_rounds) {
    std::lock_guard<std::recursive_mutex> one_persistent_solve(persist_lock(ar->device));
    StateBuffers &sb = *m.sb;
    eg_status rc = EG_OK;
    Totals tot;
    int dev = DEV_OK;
    bool exact = false, seeded = false;
    long long nproven = 0;
    // SCC-ordered solving: the levels of the condensation in turn, lowest
    // first, each a lift with cap C over its own vertices (the allocation-free
    // route has no room for the condensation and ignores the option)
    if (ar->scc_order && !m.fixed && m.attempt_only == 0 && (rc = scc_levels(ar, s)) != EG_OK) return rc;
    // a condensation of one level (one component, as on road-like grids)
    // orders nothing: such a game takes the default route with its trials
    if (ar->scc_order && !m.fixed && m.attempt_only == 0 && ar->scc_nlevels > 1) {
        for (int l = 0; l < ar->scc_nlevels && dev == DEV_OK; ++l) {
            Launch L = launch_of(ar, ar->warm_start, max_rounds);
            L.level = ar->scc_level;
            L.cur_level = l;
            rc = bits == 32 ? run_phase<int>(ar, m, sb, WeightView{scale, shift, C}, L, s, tot, EG_PHASE_LEVEL, dev)
                            : run_phase<long long>(ar, m, sb, WeightView{scale, shift, C}, L, s, tot, EG_PHASE_LEVEL,
                                                   dev);
            if (rc != EG_OK) return rc;
        }
        if (!m.in_place && (rc = enqueue_output(ar, sb, bits, credit_bits, out, s)) != EG_OK) return rc;
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        eg_status result = EG_OK;
        if (dev == DEV_TIMEOUT) {
            set_error("a device-side wait exceeded its limit");
            result = EG_ERR_TIMEOUT;
        } else if (dev == DEV_BUDGET) {
            set_error("round budget of %lld exhausted", max_rounds);
            result = EG_ERR_BUDGET;
        }
        if (st) fill_stats(st, tot, C, tot.seeded, bits, result);
        return result;
    }
    // With certification on, a first solve with cap C gets a short round
    // budget; only a game it does not finish goes through the trial caps.
    bool copied = m.in_place, attempt_out = false;
    if (m.attempt_only > 0 || (ar->cap_certify > 0 && ar->warm_start && ar->certify_after > 0 &&
                               (max_rounds == 0 || max_rounds > ar->certify_after))) {
        // the credits are copied out right behind the attempt, before the
        // host learns whether it finished; the usual case then costs one
        // synchronisation, and a game that goes on overwrites them later
        if (m.fixed) sb.dirty = true;
        const Launch L = m.attempt_only > 0 ? launch_of(ar, ar->warm_start, m.attempt_only)
                                            : launch_of(ar, 1, ar->certify_after);
        rc = bits == 32 ? launch_solve<int>(ar, sb, WeightView{scale, shift, C}, s, L)
                        : launch_solve<long long>(ar, sb, WeightView{scale, shift, C}, s, L);
        if (rc != EG_OK) return rc;
        if (!m.in_place) {
            if ((rc = enqueue_output(ar, sb, bits, credit_bits, out, s)) != EG_OK) return rc;
            attempt_out = true;
        }
        EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        add_totals(tot, ar, EG_PHASE_ATTEMPT, C);
        dev = ((const Ctrl *)ar->host_ctrl)->status;
        if (dev == DEV_OK) {
            exact = copied = true;
        } else {
            sb.dirty = true;
            if (dev == DEV_BUDGET && m.attempt_only == 0) dev = DEV_OK;
        }
        if (m.attempt_only > 0 && dev != DEV_OK) {
            set_error(dev == DEV_BUDGET ? "no fixpoint within %lld rounds" : "a device-side wait exceeded its limit",
                      m.attempt_only);
            if (st) fill_stats(st, tot, C, tot.seeded, bits, dev == DEV_BUDGET ? EG_ERR_BUDGET : EG_ERR_TIMEOUT);
            return dev == DEV_BUDGET ? EG_ERR_BUDGET : EG_ERR_TIMEOUT;
        }
    }
    bool trial_failed = false;
    if (!exact && dev == DEV_OK) {
        rc = bits == 32 ? certify<int>(ar, m, scale, shift, C, wmax, s, max_rounds, tot, dev, exact, seeded, nproven)
                        : certify<long long>(ar, m, scale, shift, C, wmax, s, max_rounds, tot, dev, exact, seeded,
                                             nproven);
        if (rc != EG_OK) return rc;
        trial_failed = dev != DEV_OK;
    }
    const bool final_launch = dev == DEV_OK && !exact;
    if (final_launch) {
        if (m.fixed) sb.dirty = true;
        Launch L = launch_of(ar, ar->warm_start, max_rounds);
        L.preseeded = seeded;  // proven losses start at TOP
        if (seeded)
            EG_CUDA_TRY(cudaMemcpyAsync(sb.d.seed_bits, m.cert_w1, ((size_t)ar->n + 31) / 32 * 4,
                                        cudaMemcpyDeviceToDevice, s));
        WeightView W{scale, shift, C};
        rc = bits == 32 ? launch_solve<int>(ar, sb, W, s, L) : launch_solve<long long>(ar, sb, W, s, L);
        if (rc != EG_OK) return rc;
    }

    // credits out (unless the first attempt's copy already holds them).  A
    // lift with cap C stopped early is below the least fixpoint everywhere;
    // a dual or capped lift stopped early bounds nothing, so then the output
    // keeps the first attempt's credits, or else becomes all zeros.
    bool zero_host = false;
    if (trial_failed) {
        if (m.in_place || !attempt_out) {
            const size_t bytes = (size_t)ar->n * ((credit_bits == 0 ? 64 : bits) / 8);
            cudaPointerAttributes attr{};
            const bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess &&
                                 (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            if (dev_out) EG_CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
            else zero_host = true;
        }
    } else if (!copied && (rc = enqueue_output(ar, sb, bits, credit_bits, out, s)) != EG_OK) {
        return rc;
    }
    if (final_launch)
        EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    if (zero_host) memset(out, 0, (size_t)ar->n * ((credit_bits == 0 ? 64 : bits) / 8));
    if (final_launch) {
        add_totals(tot, ar, tot.phases.empty() ? EG_PHASE_ATTEMPT : EG_PHASE_FINAL, C);
        dev = ((const Ctrl *)ar->host_ctrl)->status;
    }
    eg_status result = EG_OK;
    if (dev == DEV_TIMEOUT) {
        set_error("a device-side wait exceeded its limit");
        result = EG_ERR_TIMEOUT;
        sb.dirty = true;
    } else if (dev == DEV_BUDGET) {
        set_error("round budget of %lld exhausted", max_rounds);
        result = EG_ERR_BUDGET;
        sb.dirty = true;
    }
    if (st) fill_stats(st, tot, C, seeded ? nproven : tot.seeded, bits, result);
    return result;
}

eg_status solve(eg_arena *ar, int credit_bits, long long scale, long long shift, void *out, eg_stats *st,
                cudaStream_t s, long long max_rounds, long long attempt_only) {
    if (credit_bits != 0 && credit_bits != 32 && credit_bits != 64) {
        set_error("credit_bits must be 0, 32 or 64");
        return EG_ERR_INVALID;
    }
    long long sa = scale < 0 ? -scale : scale, sh = shift < 0 ? -shift : shift;
    if (sa > (1LL << 30) || sh > (1LL << 61)) {
        set_error("weight map out of range");
        return EG_ERR_INVALID;
    }
    long long C = 0, wmax = 0;
    eg_status rc = compute_bound(ar, scale, shift, &C, &wmax, s);
    if (rc != EG_OK) return rc;
    const bool fits32 = C + wmax <= 0x7fffffffLL - 1;
    int bits = credit_bits == 0 ? (fits32 ? 32 : 64) : credit_bits;
    if (bits == 32 && !fits32) {
        set_error("int32 credits cannot hold C + max|w'| = %lld", C + wmax);
        return EG_ERR_OVERFLOW;
    }
    if ((rc = ensure_state(ar, bits)) != EG_OK) return rc;
    SolveMem m;
    m.sb = bits == 32 ? &ar->st32 : &ar->st64;
    m.attempt_only = attempt_only;
    return solve_route(ar, m, bits, credit_bits, scale, shift, C, wmax, out, st, s, max_rounds);
}

}  // namespace eg

namespace eg {

// ---------------------------------------------------------------------------
// Batched solves (eg_plan).  Instances are laid out back to back in one
// credit array; a table maps each credit index to its instance's arena view.
// The solve (warm start, init, fixpoint, counter read-back) is captured once
// into a CUDA graph and replayed by every run.

struct eg_plan_impl {
    eg_arena *ar = nullptr;
    int count = 0;
    long long nf = 0;
    int bits = 32;       // computed in
    int out_bits = 64;   // written out
    std::vector<int> fbase, delta, n_of, bits_alone;
    std::vector<long long> scale, shift, C;
    void *table = nullptr;  // device instance table
    int *lut = nullptr;     // device block lookup of the instance table (non-uniform instances)
    int *d_tiles = nullptr;  // tile list of the certified trials' launches (allocated on first use)
    InstTable I{};
    StateBuffers sb;
    cudaStream_t own = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk = nullptr;
    void *host_ctrl = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long graph_rounds = -1;
    int graph_opts[6] = {-1, -1, -1, -1, -1, -1};
    long long graph_pairs = -1;
    unsigned long long graph_wait = 0;
    bool graph_failed = false;
    // certified trial caps (allocated on first use)
    std::vector<long long> wmax;  // max |w'| per instance
    void *cert_block = nullptr;
    long long *d_s2 = nullptr, *d_h2 = nullptr, *d_C2 = nullptr;
    int *d_active = nullptr, *d_busy = nullptr;
    unsigned long long *d_cnt = nullptr;
    unsigned *cert_w0 = nullptr, *cert_w1 = nullptr;
    StateBuffers sd;  // int64 state of the dual lifts
};

eg_status plan_release(eg_plan_impl *p);
static eg_status plan_destroy(eg_plan_impl *p) { return plan_release(p); }

eg_status plan_release(eg_plan_impl *p) {
    if (!p) return EG_OK;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    free_state(p->sb);
    free_state(p->sd);
    if (p->cert_block) cudaFree(p->cert_block);
    if (p->table) cudaFree(p->table);
    if (p->lut) cudaFree(p->lut);
    if (p->d_tiles) cudaFree(p->d_tiles);
    if (p->own) cudaStreamDestroy(p->own);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->evk) cudaEventDestroy(p->evk);
    if (p->host_ctrl) cudaFreeHost(p->host_ctrl);
    delete p;
    return EG_OK;
}

eg_status plan_create(eg_arena *ar, int count, const int32_t *part, const int64_t *w_scale, const int64_t *w_shift,
                      int credit_bits, eg_plan_impl **out) {
    *out = nullptr;
    if (count < 1) {
        set_error("count must be >= 1");
        return EG_ERR_INVALID;
    }
    if (credit_bits != 0 && credit_bits != 32 && credit_bits != 64) {
        set_error("credit_bits must be 0, 32 or 64");
        return EG_ERR_INVALID;
    }
    std::vector<long long> pp = ar->part_ptr;
    if (pp.empty()) pp = {0, (long long)ar->n};
    const int parts = (int)pp.size() - 1;
    eg_plan_impl *p = new (std::nothrow) eg_plan_impl();
    if (!p) {
        set_error("host allocation failed");
        return EG_ERR_OOM;
    }
    p->ar = ar;
    p->count = count;
    p->fbase.resize(count + 1);
    p->delta.resize(count);
    p->n_of.resize(count);
    p->scale.resize(count);
    p->shift.resize(count);
    long long nf = 0;
    for (int i = 0; i < count; ++i) {
        const int k = part ? part[i] : i;
        if (k < 0 || k >= parts) {
            set_error("instance %d names game %d of %d", i, k, parts);
            plan_destroy(p);
            return EG_ERR_INVALID;
        }
        const long long sc = w_scale ? w_scale[i] : 1, sh = w_shift ? w_shift[i] : 0;
        if ((sc < 0 ? -sc : sc) > (1LL << 30) || (sh < 0 ? -sh : sh) > (1LL << 61)) {
            set_error("weight map of instance %d out of range", i);
            plan_destroy(p);
            return EG_ERR_INVALID;
        }
        p->fbase[i] = (int)nf;
        p->delta[i] = (int)(nf - pp[k]);
        p->n_of[i] = (int)(pp[k + 1] - pp[k]);
        p->scale[i] = sc;
        p->shift[i] = sh;
        nf += pp[k + 1] - pp[k];
        if (nf >= (1LL << 31) - 1) {
            set_error("instances hold more than 2^31 - 1 credits");
            plan_destroy(p);
            return EG_ERR_INVALID;
        }
    }
    p->fbase[count] = (int)nf;
    p->nf = nf;
    cudaStream_t s = nullptr;
#define PTRY(expr)                                                          \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) {                                            \
            set_error("%s failed: %s", #expr, cudaGetErrorString(_e));      \
            plan_destroy(p);                                                \
            return _e == cudaErrorMemoryAllocation ? EG_ERR_OOM : EG_ERR_CUDA; \
        }                                                                   \
    } while (0)
    PTRY(cudaStreamCreateWithFlags(&p->own, cudaStreamNonBlocking));
    s = p->own;
    PTRY(cudaEventCreate(&p->ev0));
    PTRY(cudaEventCreate(&p->ev1));
    PTRY(cudaEventCreate(&p->evk));
    PTRY(cudaMallocHost(&p->host_ctrl, sizeof(Ctrl)));
    // device table: fbase (count+1 ints), delta (count ints), scale, shift, C (count long longs), and
    // per-instance bound accumulators
    const size_t ints = (size_t)2 * count + 1;
    const size_t off_ll = ((ints * 4 + 15) / 16) * 16;
    const size_t bytes = off_ll + (size_t)5 * count * 8;
    char *tb = nullptr;
    PTRY(cudaMalloc((void **)&tb, bytes));
    p->table = tb;
    int *d_fbase = (int *)tb, *d_delta = d_fbase + count + 1;
    long long *d_scale = (long long *)(tb + off_ll), *d_shift = d_scale + count, *d_C = d_shift + count;
    unsigned long long *d_accC = (unsigned long long *)(d_C + count), *d_accW = d_accC + count;
    PTRY(cudaMemcpyAsync(d_fbase, p->fbase.data(), (count + 1) * 4, cudaMemcpyHostToDevice, s));
    PTRY(cudaMemcpyAsync(d_delta, p->delta.data(), count * 4, cudaMemcpyHostToDevice, s));
    PTRY(cudaMemcpyAsync(d_scale, p->scale.data(), count * 8, cudaMemcpyHostToDevice, s));
    PTRY(cudaMemcpyAsync(d_shift, p->shift.data(), count * 8, cudaMemcpyHostToDevice, s));
    PTRY(cudaMemsetAsync(d_accC, 0, (size_t)2 * count * 8, s));
    int uniform = p->n_of[0];
    for (int i = 1; i < count; ++i)
        if (p->n_of[i] != uniform) uniform = 0;
    p->I = InstTable{count, uniform, d_fbase, d_delta, d_scale, d_shift, d_C};
    if (!uniform) {
        // block lookup of the instance of a credit: blocks of 2^shift credits,
        // no longer than the shortest instance, so at most one step past it
        int min_n = p->n_of[0];
        for (int i = 1; i < count; ++i) min_n = std::min(min_n, p->n_of[i]);
        int shift = 0;
        while (shift < 20 && (2 << shift) <= min_n) ++shift;
        const size_t blocks = (size_t)(nf >> shift) + 1;
        std::vector<int> lut(blocks);
        int i = 0;
        for (size_t b = 0; b < blocks; ++b) {
            const long long x = (long long)b << shift;
            while (i + 1 < count && p->fbase[i + 1] <= x) ++i;
            lut[b] = i;
        }
        PTRY(cudaMalloc((void **)&p->lut, blocks * 4));
        PTRY(cudaMemcpyAsync(p->lut, lut.data(), blocks * 4, cudaMemcpyHostToDevice, s));
        PTRY(cudaStreamSynchronize(s));
        p->I.lut = p->lut;
        p->I.lut_shift = shift;
    }
    const int sms = num_sms(ar->device);
    k_bound_inst<<<(int)std::min<long long>((nf + 255) / 256, (long long)sms * 32), 256, 0, s>>>(
        ar->d, p->I, (int)nf, d_accC, d_accW);
    PTRY(cudaGetLastError());
    std::vector<unsigned long long> hc(2 * (size_t)count);
    PTRY(cudaMemcpyAsync(hc.data(), d_accC, (size_t)2 * count * 8, cudaMemcpyDeviceToHost, s));
    PTRY(cudaStreamSynchronize(s));
    p->C.resize(count);
    p->wmax.resize(count);
    p->bits_alone.resize(count);
    bool all32 = true;
    for (int i = 0; i < count; ++i) {
        p->C[i] = (long long)hc[i];
        p->wmax[i] = (long long)hc[count + i];
        const bool fits = (long long)hc[i] + (long long)hc[count + i] <= 0x7fffffffLL - 1;
        p->bits_alone[i] = fits ? 32 : 64;
        all32 = all32 && fits;
    }
    if (credit_bits == 32 && !all32) {
        set_error("int32 credits cannot hold every instance");
        plan_destroy(p);
        return EG_ERR_OVERFLOW;
    }
    p->bits = (credit_bits == 64 || !all32) ? 64 : 32;
    p->out_bits = credit_bits == 32 ? 32 : 64;
    PTRY(cudaMemcpyAsync(d_C, p->C.data(), count * 8, cudaMemcpyHostToDevice, s));
    eg_status rc = alloc_state(p->sb, nf, p->bits);
    if (rc != EG_OK) {
        plan_destroy(p);
        return rc;
    }
    PTRY(cudaStreamSynchronize(s));
#undef PTRY
    *out = p;
    return EG_OK;
}

// Enqueues one batched solve on s (also used under stream capture).
static eg_status plan_enqueue(eg_plan_impl *p, const Launch &L, cudaStream_t s, cudaEvent_t evk) {
    WeightView W{1, 0, 0};
    eg_status rc = p->bits == 32
                       ? enqueue_solve<true, int>(p->ar->d, W, p->I, p->nf, p->sb, L, p->ar->device, s, evk)
                       : enqueue_solve<true, long long>(p->ar->d, W, p->I, p->nf, p->sb, L, p->ar->device, s, evk);
    if (rc != EG_OK) return rc;
    EG_CUDA_TRY(cudaMemcpyAsync(p->host_ctrl, p->sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    return EG_OK;
}

void plan_instance_info(const eg_plan_impl *p, int i, long long *offset, long long *n, long long *C, int *bits) {
    if (offset) *offset = p->fbase[i];
    if (n) *n = p->n_of[i];
    if (C) *C = p->C[i];
    if (bits) *bits = p->bits_alone[i];
}

// Counters of the plan's last launch; a graph replay has no event right
// before its fixpoint kernel, so its kernel time is the whole replay's.  The
// caps differ per instance: the phase records carry 0.
static void plan_add_totals(Totals &t, const eg_plan_impl *p, bool kernel_event, int kind) {
    float ms = 0.f, kms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    if (kernel_event) cudaEventElapsedTime(&kms, p->evk, p->ev1);
    add_launch(t, (const Ctrl *)p->host_ctrl, ms, kernel_event ? kms : ms, kind, 0);
}

// One batched solve over the instances of I (direct launches), run to its end.
template <typename T>
static eg_status plan_phase(eg_plan_impl *p, StateBuffers &sb, const InstTable &I, const Launch &L, cudaStream_t s,
                            Totals &t, int kind, int &dev) {
    EG_CUDA_TRY(cudaEventRecord(p->ev0, s));
    eg_status rc = enqueue_solve<true, T>(p->ar->d, WeightView{1, 0, 0}, I, p->nf, sb, L, p->ar->device, s, p->evk);
    if (rc != EG_OK) return rc;
    EG_CUDA_TRY(cudaEventRecord(p->ev1, s));
    EG_CUDA_TRY(cudaMemcpyAsync(p->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    plan_add_totals(t, p, true, kind);
    dev = ((const Ctrl *)p->host_ctrl)->status;
    if (dev != DEV_OK) sb.dirty = true;
    return EG_OK;
}

// Certified trial caps per instance (the single solve's trials, per
// instance): instances the budgeted first attempt finished are exact; every
// other one runs capped and dual lifts with its own B and K until it is
// decided, and is then left as it is by the later launches.  What no trial
// decides ends with cap C from its proven TOP starts.
template <typename T>
static eg_status plan_certify(eg_plan_impl *p, cudaStream_t s, long long max_rounds, Totals &t, int &dev) {
    eg_arena *ar = p->ar;
    const int cnt = p->count;
    const long long nf = p->nf;
    const size_t words = ((size_t)nf + 31) / 32, bm = align_up(words * 4);
    if (!p->cert_block) {
        const size_t o_h2 = align_up((size_t)cnt * 8), o_C2 = o_h2 + align_up((size_t)cnt * 8);
        const size_t o_act = o_C2 + align_up((size_t)cnt * 8), o_busy = o_act + align_up((size_t)cnt * 4);
        const size_t o_cnt = o_busy + align_up((size_t)cnt * 4), o_w0 = o_cnt + align_up((size_t)cnt * 8);
        const size_t bytes = o_w0 + 2 * bm;
        char *b = nullptr;
        EG_CUDA_TRY(cudaMalloc((void **)&b, bytes));
        p->cert_block = b;
        p->d_s2 = (long long *)b;
        p->d_h2 = (long long *)(b + o_h2);
        p->d_C2 = (long long *)(b + o_C2);
        p->d_active = (int *)(b + o_act);
        p->d_busy = (int *)(b + o_busy);
        p->d_cnt = (unsigned long long *)(b + o_cnt);
        p->cert_w0 = (unsigned *)(b + o_w0);
        p->cert_w1 = (unsigned *)(b + o_w0 + bm);
    }
    // instances with no entry left in the lists are finished, hence exact
    const int r = (int)((const Ctrl *)p->host_ctrl)->r_next;
    EG_CUDA_TRY(cudaMemsetAsync(p->d_busy, 0, (size_t)cnt * 4, s));
    const int sms = num_sms(ar->device);
    k_busy_plan<<<sms * 4, 256, 0, s>>>(p->sb.d.ctrl, r % 3, p->sb.d.pull_items[r & 1], p->sb.d.push_items[r & 1],
                                        p->I, p->d_busy);
    EG_CUDA_TRY(cudaGetLastError());
    std::vector<int> act(cnt, 0);
    EG_CUDA_TRY(cudaMemcpyAsync(act.data(), p->d_busy, (size_t)cnt * 4, cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    p->sb.dirty = true;
    int nact = 0;
    for (int i = 0; i < cnt; ++i) nact += act[i] != 0;
    if (nact == 0) return EG_OK;
    if (p->sd.bits != 64 || p->sd.nf != nf) {
        eg_status rc = alloc_state(p->sd, nf, 64);
        if (rc != EG_OK) return rc;
    }
    EG_CUDA_TRY(cudaMemsetAsync(p->cert_w0, 0, 2 * bm, s));
    constexpr long long LIM = 1LL << 61;
    const long long raw = std::max(1LL, ar->wmax_plain), mult = ar->cap_certify;
    std::vector<long long> B(cnt, 0), K(cnt, 0), hs(cnt), hh(cnt), hC(cnt);
    std::vector<int> direct(cnt, 0), skip(cnt, 0), on(cnt, 0), dual_on(cnt, 0);
    std::vector<unsigned long long> und(cnt);
    auto fits = [&](int i) {
        const long long inner = (p->scale[i] < 0 ? -p->scale[i] : p->scale[i]) * raw +
                                (p->shift[i] < 0 ? -p->shift[i] : p->shift[i]) + 1;
        return K[i] <= LIM / inner && B[i] <= LIM / (K[i] + 1);
    };
    for (int i = 0; i < cnt; ++i) {
        if (!act[i]) continue;
        const long long wm = std::max(1LL, p->wmax[i]);
        if (wm > LIM / 4 / mult) {
            skip[i] = 1;
            continue;
        }
        B[i] = mult * wm;
        K[i] = std::min((long long)ar->dual_k, (long long)p->n_of[i] + 1);
        if (B[i] >= p->C[i]) direct[i] = 1;  // cap C: the capped lift is the exact one
        else if (!fits(i)) skip[i] = 1;
    }
    InstTable It = p->I;
    It.scale = p->d_s2;
    It.shift = p->d_h2;
    It.C = p->d_C2;
    It.active = p->d_active;
    // the tiles covering the instances of the set uploaded last (see
    // tile_count), when they hold under half of the credits; else every tile
    std::vector<int> htiles;
    const int *cur_tiles = nullptr;
    long long cur_ntiles = 0;
    auto select_tiles = [&](const std::vector<int> &a) -> eg_status {
        long long sel = 0;
        for (int i = 0; i < cnt; ++i)
            if (a[i]) sel += p->n_of[i];
        cur_tiles = nullptr;
        cur_ntiles = 0;
        if (2 * sel >= nf) return EG_OK;
        htiles.clear();
        for (int i = 0; i < cnt; ++i) {
            if (!a[i] || p->n_of[i] == 0) continue;
            int t0 = p->fbase[i] >> 5;
            const int t1 = (p->fbase[i + 1] - 1) >> 5;
            if (!htiles.empty() && htiles.back() >= t0) t0 = htiles.back() + 1;
            for (int t = t0; t <= t1; ++t) htiles.push_back(t);
        }
        if (!p->d_tiles) EG_CUDA_TRY(cudaMalloc((void **)&p->d_tiles, ((size_t)(nf + 31) / 32 + 1) * 4));
        if (!htiles.empty())
            EG_CUDA_TRY(cudaMemcpyAsync(p->d_tiles, htiles.data(), htiles.size() * 4, cudaMemcpyHostToDevice, s));
        cur_tiles = p->d_tiles;
        cur_ntiles = (long long)htiles.size();
        return EG_OK;
    };
    auto upload = [&](const std::vector<int> &a) -> eg_status {
        eg_status trc = select_tiles(a);
        if (trc != EG_OK) return trc;
        EG_CUDA_TRY(cudaMemcpyAsync(p->d_s2, hs.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync(p->d_h2, hh.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync(p->d_C2, hC.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync(p->d_active, a.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors change before the next upload
        return EG_OK;
    };
    // und[i] = credits of instance i at TOP in the capped fixpoint without a proof of loss
    auto count = [&]() -> eg_status {
        EG_CUDA_TRY(cudaMemsetAsync(p->d_cnt, 0, (size_t)cnt * 8, s));
        k_count_undecided_inst<T><<<wblocks_of(nf, sms), 256, 0, s>>>((const T *)p->sb.d.f, p->cert_w1, p->I,
                                                                      (int)nf, p->d_cnt, cur_tiles, cur_ntiles);
        EG_CUDA_TRY(cudaGetLastError());
        EG_CUDA_TRY(cudaMemcpyAsync(und.data(), p->d_cnt, (size_t)cnt * 8, cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        return EG_OK;
    };
    const int wblocks = wblocks_of(nf, sms);
    eg_status rc = EG_OK;
    for (int k = 0; k < CERT_TRIALS; ++k) {
        int ntrial = 0;
        for (int i = 0; i < cnt; ++i) {
            on[i] = act[i] && !skip[i];
            ntrial += on[i];
        }
        if (ntrial == 0) break;
        t.trials = k + 1;
        // the game's lifts with cap B (cap C for the direct ones): proven
        // player-1 vertices start at TOP
        for (int i = 0; i < cnt; ++i) {
            hs[i] = p->scale[i];
            hh[i] = p->shift[i];
            hC[i] = on[i] && !direct[i] ? B[i] : p->C[i];
        }
        if ((rc = upload(on)) != EG_OK) return rc;
        EG_CUDA_TRY(cudaMemcpyAsync(p->sb.d.seed_bits, p->cert_w1, words * 4, cudaMemcpyDeviceToDevice, s));
        Launch Lp = launch_of(ar, 1, max_rounds);
        Lp.preseeded = true;
        Lp.tiles = cur_tiles;
        Lp.ntiles = cur_ntiles;
        rc = plan_phase<T>(p, p->sb, It, Lp, s, t, EG_PHASE_CAPPED, dev);
        if (rc != EG_OK || dev != DEV_OK) return rc;
        k_or_bits<<<(int)std::min<size_t>((words + 255) / 256, 1024), 256, 0, s>>>(p->cert_w1, p->sb.d.seed_bits,
                                                                                   (int)words);
        k_mark_finite<T><<<wblocks, 256, 0, s>>>((const T *)p->sb.d.f, (int)nf, p->cert_w0, It, cur_tiles,
                                                 cur_ntiles);
        EG_CUDA_TRY(cudaGetLastError());
        if ((rc = count()) != EG_OK) return rc;
        int ndual = 0;
        for (int i = 0; i < cnt; ++i) {
            dual_on[i] = 0;
            if (!on[i]) continue;
            if (direct[i] || und[i] == 0) {
                act[i] = 0;  // exact: later launches leave it as it is
                continue;
            }
            dual_on[i] = 1;
            ++ndual;
        }
        if (ndual > 0) {
            // dual lifts: owners swapped, weights -(K w' + 1), cap (K + 1) B;
            // proven player-0 vertices start at TOP, proven player-1 ones are held at 0
            for (int i = 0; i < cnt; ++i) {
                hs[i] = dual_on[i] ? -K[i] * p->scale[i] : p->scale[i];
                hh[i] = dual_on[i] ? 1 - K[i] * p->shift[i] : p->shift[i];
                hC[i] = dual_on[i] ? (K[i] + 1) * B[i] : p->C[i];
            }
            if ((rc = upload(dual_on)) != EG_OK) return rc;
            EG_CUDA_TRY(cudaMemcpyAsync(p->sd.d.seed_bits, p->cert_w0, words * 4, cudaMemcpyDeviceToDevice, s));
            Launch Ld = launch_of(ar, 1, max_rounds);
            Ld.inv = 1;
            Ld.preseeded = true;
            Ld.frozen = p->cert_w1;
            Ld.tiles = cur_tiles;
            Ld.ntiles = cur_ntiles;
            rc = plan_phase<long long>(p, p->sd, It, Ld, s, t, EG_PHASE_DUAL, dev);
            if (rc != EG_OK || dev != DEV_OK) return rc;
            k_mark_finite<long long><<<wblocks, 256, 0, s>>>((const long long *)p->sd.d.f, (int)nf, p->cert_w1, It,
                                                             cur_tiles, cur_ntiles);
            EG_CUDA_TRY(cudaGetLastError());
            if ((rc = count()) != EG_OK) return rc;
            for (int i = 0; i < cnt; ++i)
                if (dual_on[i] && und[i] == 0) act[i] = 0;  // the capped fixpoint is exact
        }
        for (int i = 0; i < cnt; ++i) {
            if (!on[i] || !act[i]) continue;
            if (B[i] > LIM / 4) {
                skip[i] = 1;
                continue;
            }
            B[i] *= 4;
            K[i] = std::min(K[i] * 8, (long long)p->n_of[i] + 1);
            if (B[i] >= p->C[i]) direct[i] = 1;
            else if (!fits(i)) skip[i] = 1;
        }
    }
    int left = 0;
    for (int i = 0; i < cnt; ++i) left += act[i] != 0;
    if (left == 0) return EG_OK;
    // cap C from the proven TOP starts for whatever no trial decided
    for (int i = 0; i < cnt; ++i) {
        hs[i] = p->scale[i];
        hh[i] = p->shift[i];
        hC[i] = p->C[i];
    }
    if ((rc = upload(act)) != EG_OK) return rc;
    EG_CUDA_TRY(cudaMemcpyAsync(p->sb.d.seed_bits, p->cert_w1, words * 4, cudaMemcpyDeviceToDevice, s));
    Launch Lf = launch_of(ar, 1, max_rounds);
    Lf.preseeded = true;
    Lf.tiles = cur_tiles;
    Lf.ntiles = cur_ntiles;
    return plan_phase<T>(p, p->sb, It, Lf, s, t, EG_PHASE_FINAL, dev);
}

eg_status plan_run(eg_plan_impl *p, void *out, eg_stats *st, cudaStream_t user, long long max_rounds) {
    eg_arena *ar = p->ar;
    std::lock_guard<std::recursive_mutex> one_persistent_solve(persist_lock(ar->device));
    // with certification on, the first batched solve gets a short round
    // budget, and only the instances it does not finish go through the trials
    const bool cert = ar->cap_certify > 0 && ar->warm_start && ar->certify_after > 0 &&
                      (max_rounds == 0 || max_rounds > ar->certify_after);
    const Launch L = launch_of(ar, ar->warm_start, cert ? ar->certify_after : max_rounds);
    cudaStream_t s = user ? user : p->own;
    // scratch left dirty by an aborted run is reset outside the graph
    if (p->sb.dirty) {
        const int sms = num_sms(ar->device);
        if (p->bits == 32) k_fill<int><<<sms * 4, 256, 0, s>>>((int *)p->sb.d.acc, p->nf, Cred<int>::TOP);
        else k_fill<long long><<<sms * 4, 256, 0, s>>>((long long *)p->sb.d.acc, p->nf, Cred<long long>::TOP);
        EG_CUDA_TRY(cudaMemsetAsync(p->sb.d.acc_done, 0, (size_t)p->nf * 4, s));
        for (int k = 0; k < 2; ++k) {
            EG_CUDA_TRY(cudaMemsetAsync(p->sb.d.bits_pull[k], 0, ((size_t)p->nf + 31) / 32 * 4, s));
            EG_CUDA_TRY(cudaMemsetAsync(p->sb.d.bits_push[k], 0, ((size_t)p->nf + 31) / 32 * 4, s));
        }
        p->sb.dirty = false;
    }
    const bool same = p->graph && p->graph_rounds == L.max_rounds && p->graph_opts[0] == L.local_windows &&
                      p->graph_opts[1] == L.local_maxdeg && p->graph_opts[2] == L.warm_start &&
                      p->graph_opts[3] == L.blocks_per_sm && p->graph_opts[4] == L.chunk_edges &&
                      p->graph_opts[5] == L.sweeps &&
                      p->graph_pairs == L.seed_max_pairs &&
                      p->graph_wait == L.wait_ns;
    if (!ar->use_graph && p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    if (ar->use_graph && !same && !p->graph_failed) {
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(p->own, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            eg_status rc = plan_enqueue(p, L, p->own, nullptr);
            ok = cudaStreamEndCapture(p->own, &g) == cudaSuccess && rc == EG_OK && g;
        }
        if (ok) ok = cudaGraphInstantiate(&p->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (ok) {
            p->graph_rounds = L.max_rounds;
            p->graph_opts[0] = L.local_windows;
            p->graph_opts[1] = L.local_maxdeg;
            p->graph_opts[2] = L.warm_start;
            p->graph_opts[3] = L.blocks_per_sm;
            p->graph_opts[4] = L.chunk_edges;
            p->graph_opts[5] = L.sweeps;
            p->graph_pairs = L.seed_max_pairs;
            p->graph_wait = L.wait_ns;
        } else {
            p->graph = nullptr;
            p->graph_failed = true;  // capture unsupported here: launch directly from now on
        }
    }
    EG_CUDA_TRY(cudaEventRecord(p->ev0, s));
    if (p->graph) {
        EG_CUDA_TRY(cudaGraphLaunch(p->graph, s));
    } else {
        eg_status rc = plan_enqueue(p, L, s, p->evk);
        if (rc != EG_OK) return rc;
    }
    EG_CUDA_TRY(cudaEventRecord(p->ev1, s));
    Totals tot;
    int dev = DEV_OK;
    if (cert) {
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        plan_add_totals(tot, p, p->graph == nullptr, EG_PHASE_ATTEMPT);
        dev = ((const Ctrl *)p->host_ctrl)->status;
        if (dev == DEV_BUDGET) {
            eg_status rc = p->bits == 32 ? plan_certify<int>(p, s, max_rounds, tot, dev)
                                         : plan_certify<long long>(p, s, max_rounds, tot, dev);
            if (rc != EG_OK) return rc;
        }
    }
    // credits out; a dual or capped lift stopped early bounds nothing from
    // below, so then the output is all zeros (below every fixpoint)
    cudaPointerAttributes attr{};
    const bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess &&
                         (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    const bool trial_failed = cert && dev != DEV_OK && !tot.phases.empty() &&
                              (tot.phases.back().kind == EG_PHASE_DUAL || tot.phases.back().kind == EG_PHASE_CAPPED);
    const size_t out_bytes = (size_t)p->nf * (p->out_bits / 8);
    if (trial_failed) {
        if (dev_out) EG_CUDA_TRY(cudaMemsetAsync(out, 0, out_bytes, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        if (!dev_out) memset(out, 0, out_bytes);
    }
    void *src = p->sb.d.f, *tmp = nullptr;
    if (!trial_failed && p->out_bits != p->bits) {
        EG_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)p->nf * 8, s));
        k_widen<<<(int)std::min<long long>((p->nf + 255) / 256, 4096), 256, 0, s>>>((const int *)p->sb.d.f,
                                                                                    (long long *)tmp, (int)p->nf);
        EG_CUDA_TRY(cudaGetLastError());
        src = tmp;
    }
    if (!trial_failed)
        EG_CUDA_TRY(cudaMemcpyAsync(out, src, out_bytes, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    s));
    if (tmp) EG_CUDA_TRY(cudaFreeAsync(tmp, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    if (!cert) {
        plan_add_totals(tot, p, p->graph == nullptr, EG_PHASE_ATTEMPT);
        dev = ((const Ctrl *)p->host_ctrl)->status;
    }
    eg_status result = EG_OK;
    if (dev == DEV_TIMEOUT) {
        set_error("a device-side wait exceeded its limit");
        result = EG_ERR_TIMEOUT;
        p->sb.dirty = true;
    } else if (dev == DEV_BUDGET) {
        set_error("round budget of %lld exhausted", max_rounds);
        result = EG_ERR_BUDGET;
        p->sb.dirty = true;
    }
    if (st) {
        long long cmax = 0;
        for (long long c : p->C) cmax = std::max(cmax, c);
        fill_stats(st, tot, cmax, tot.seeded, p->bits, result);
        if (p->graph) st->fixpoint_ms = -1.0;
    }
    return result;
}

}  // namespace eg

struct eg_plan : eg::eg_plan_impl {};

namespace eg {
eg_plan_impl *plan_impl(eg_plan *plan) { return plan; }
eg_arena *plan_arena(const eg_plan_impl *p) { return p->ar; }
int plan_count(const eg_plan_impl *p) { return p->count; }
int plan_bits(const eg_plan_impl *p) { return p->bits; }
}  // namespace eg

extern "C" {

eg_status eg_plan_create(eg_arena *arena, int32_t count, const int32_t *part, const int64_t *w_scale,
                         const int64_t *w_shift, int32_t credit_bits, eg_plan **out) {
    eg::clear_error();
    if (!arena || !out) {
        eg::set_error("arena and out are required");
        return EG_ERR_INVALID;
    }
    eg::eg_plan_impl *p = nullptr;
    eg_status rc = eg::plan_create(arena, count, part, w_scale, w_shift, credit_bits, &p);
    *out = (eg_plan *)p;
    return rc;
}

eg_status eg_plan_instance(eg_plan *plan, int32_t i, int64_t *offset, int64_t *n, int64_t *C, int32_t *bits) {
    eg::clear_error();
    if (!plan || i < 0 || i >= plan->count) {
        eg::set_error("no such instance");
        return EG_ERR_INVALID;
    }
    if (offset) *offset = plan->fbase[i];
    if (n) *n = plan->n_of[i];
    if (C) *C = plan->C[i];
    if (bits) *bits = plan->bits_alone[i];
    return EG_OK;
}

eg_status eg_plan_run(eg_plan *plan, void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds) {
    eg::clear_error();
    if (!plan || !credits_out) {
        eg::set_error("plan and credits_out are required");
        return EG_ERR_INVALID;
    }
    return eg::plan_run(plan, credits_out, st, (cudaStream_t)cuda_stream, max_rounds);
}

eg_status eg_plan_destroy(eg_plan *plan) {
    eg::clear_error();
    return eg::plan_destroy(plan);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Resident solve: the state of one persistent solve over a pool of games
// that join and leave between slices of rounds (continuous batching).

namespace eg {

// Clears bits [g0, g0 + n) of a bitmap.
__global__ void k_clear_bits(unsigned *bits, int g0, int n) {
    const int w0 = g0 >> 5, w1 = (g0 + n + 31) >> 5;
    for (int w = w0 + blockIdx.x * blockDim.x + threadIdx.x; w < w1; w += gridDim.x * blockDim.x) {
        const int lo = max(g0, w << 5) - (w << 5), hi = min(g0 + n, (w + 1) << 5) - (w << 5);
        const unsigned mask = hi - lo == 32 ? FULL : (((1u << (hi - lo)) - 1u) << lo);
        atomicAnd(bits + w, ~mask);
    }
}

// Marks the instance of every entry of the pull and push lists of round r.
__global__ void k_busy(const Ctrl *c, int slot, const int *pull_items, const int *push_items, const int *inst_id,
                       int *busy) {
    const int np = (int)(ld_cg(&c->pull_ctr[slot]) & 0xffffffffu);
    const int nq = (int)(ld_cg(&c->push_ctr[slot]) & 0xffffffffu);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np + nq; i += gridDim.x * blockDim.x) {
        const int g = (i < np ? ld_cg(pull_items + i) : ld_cg(push_items + (i - np))) & 0x7fffffff;
        busy[__ldg(inst_id + g)] = 1;
    }
}

static Args<long long> resident_args(const Resident &R) {
    Args<long long> a;
    a.A = R.A;
    a.W = WeightView{1, 0, 0};
    a.I = InstTable{R.slots, 0, nullptr, R.delta, R.scale, R.shift, R.C, R.inst_id};
    a.nf = R.cap;
    a.f = (long long *)R.sb.d.f;
    for (int k = 0; k < 2; ++k) {
        a.pull_items[k] = R.sb.d.pull_items[k];
        a.pull_offs[k] = R.sb.d.pull_offs[k];
        a.push_items[k] = R.sb.d.push_items[k];
        a.push_offs[k] = R.sb.d.push_offs[k];
        a.bits_pull[k] = R.sb.d.bits_pull[k];
        a.bits_push[k] = R.sb.d.bits_push[k];
    }
    a.seed_bits = R.sb.d.seed_bits;
    a.frozen = nullptr;
    a.inv = 0;
    a.acc = (long long *)R.sb.d.acc;
    a.acc_done = R.sb.d.acc_done;
    a.ctrl = R.sb.d.ctrl;
    a.max_rounds = 0;
    a.r0 = R.r;
    a.slice = 1;
    a.doorbell = R.bell_dev;
    a.local_windows = R.local_windows;
    a.local_maxdeg = R.local_maxdeg;
    a.chunk = R.chunk_edges;
    a.wait_ns = BARRIER_LIMIT_NS;
    a.level = nullptr;
    a.cur_level = 0;
    a.tiles = nullptr;
    a.ntiles = 0;
    return a;
}

eg_status resident_reset(Resident &R, cudaStream_t s) {
    const int sms = num_sms(R.device);
    const size_t words = ((size_t)R.cap + 31) / 32;
    k_fill<long long><<<sms * 4, 256, 0, s>>>((long long *)R.sb.d.acc, R.cap, Cred<long long>::TOP);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemsetAsync(R.sb.d.acc_done, 0, (size_t)R.cap * 4, s));
    for (int k = 0; k < 2; ++k) {
        EG_CUDA_TRY(cudaMemsetAsync(R.sb.d.bits_pull[k], 0, words * 4, s));
        EG_CUDA_TRY(cudaMemsetAsync(R.sb.d.bits_push[k], 0, words * 4, s));
    }
    EG_CUDA_TRY(cudaMemsetAsync(R.sb.d.seed_bits, 0, words * 4, s));
    EG_CUDA_TRY(cudaMemsetAsync(R.sb.d.ctrl, 0, sizeof(Ctrl), s));
    R.sb.dirty = false;
    R.r = 0;
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    return EG_OK;
}

eg_status resident_create(Resident &R, int device, int cap, int slots, cudaStream_t s) {
    R.device = device;
    R.cap = cap;
    R.slots = slots;
    eg_status rc = alloc_state(R.sb, cap, 64);
    if (rc != EG_OK) return rc;
    const size_t o_busy = align_up((size_t)cap * 4), o_delta = o_busy + align_up((size_t)slots * 4);
    const size_t o_scale = o_delta + align_up((size_t)slots * 4), o_shift = o_scale + align_up((size_t)slots * 8);
    const size_t o_C = o_shift + align_up((size_t)slots * 8), bytes = o_C + align_up((size_t)slots * 8);
    char *blk = nullptr;
    EG_CUDA_TRY(cudaMalloc((void **)&blk, bytes));
    R.block = blk;
    R.inst_id = (int *)blk;
    R.busy = (int *)(blk + o_busy);
    R.delta = (int *)(blk + o_delta);
    R.scale = (long long *)(blk + o_scale);
    R.shift = (long long *)(blk + o_shift);
    R.C = (long long *)(blk + o_C);
    EG_CUDA_TRY(cudaMemsetAsync(blk, 0, bytes, s));
    EG_CUDA_TRY(cudaHostAlloc((void **)&R.bell_host, sizeof(unsigned), cudaHostAllocMapped));
    *(volatile unsigned *)R.bell_host = 0;
    EG_CUDA_TRY(cudaHostGetDevicePointer((void **)&R.bell_dev, R.bell_host, 0));
    EG_CUDA_TRY(cudaMallocHost(&R.host_ctrl, sizeof(Ctrl)));
    EG_CUDA_TRY(cudaMallocHost((void **)&R.host_busy, (size_t)slots * 4));
    EG_CUDA_TRY(cudaMallocHost((void **)&R.host_tab, (size_t)slots * 3 * 8));
    return resident_reset(R, s);
}

void resident_free(Resident &R) {
    free_state(R.sb);
    if (R.block) cudaFree(R.block);
    if (R.bell_host) cudaFreeHost(R.bell_host);
    if (R.host_ctrl) cudaFreeHost(R.host_ctrl);
    if (R.host_busy) cudaFreeHost(R.host_busy);
    if (R.host_tab) cudaFreeHost(R.host_tab);
    R.host_tab = nullptr;
    R.block = nullptr;
    R.bell_host = nullptr;
    R.host_ctrl = nullptr;
    R.host_busy = nullptr;
}

eg_status resident_admit(Resident &R, int slot, int g0, int n, long long scale, long long shift, long long C,
                         cudaStream_t s) {
    // staged in pinned memory, so the copies stay asynchronous; a slot's entry
    // is rewritten only after the slot was freed, i.e. after a synchronised slice
    long long *tab = R.host_tab + 3 * slot;
    tab[0] = scale;
    tab[1] = shift;
    tab[2] = C;
    EG_CUDA_TRY(cudaMemcpyAsync(R.scale + slot, tab + 0, 8, cudaMemcpyHostToDevice, s));
    EG_CUDA_TRY(cudaMemcpyAsync(R.shift + slot, tab + 1, 8, cudaMemcpyHostToDevice, s));
    EG_CUDA_TRY(cudaMemcpyAsync(R.C + slot, tab + 2, 8, cudaMemcpyHostToDevice, s));
    const int sms = num_sms(R.device);
    const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sms * 8);
    k_fill<int><<<blocks, 256, 0, s>>>(R.inst_id + g0, n, slot);
    k_clear_bits<<<std::max(1, std::min((n / 32 + 255) / 256 + 1, sms * 4)), 256, 0, s>>>(R.sb.d.seed_bits, g0, n);
    EG_CUDA_TRY(cudaGetLastError());
    Args<long long> a = resident_args(R);
    a.seed_bits = nullptr;
    const int sblocks = (int)std::min<long long>((n + 7) / 8, (long long)sms * 32);
    k_seed<true, long long><<<sblocks, 256, 0, s>>>(a, R.seed_max_pairs, R.sb.d.seed_bits, &R.sb.d.ctrl->seeded, g0,
                                                    g0 + n);
    EG_CUDA_TRY(cudaGetLastError());
    a.seed_bits = R.sb.d.seed_bits;
    const int r = (int)R.r;
    const int iblocks = (int)std::min<long long>((n + THREADS - 1) / THREADS, (long long)sms * 16);
    k_init<true, long long><<<iblocks, THREADS, 0, s>>>(a, g0, g0 + n, r % 3, r & 1, 1);
    EG_CUDA_TRY(cudaGetLastError());
    return EG_OK;
}

eg_status resident_slice(Resident &R, long long rounds, cudaStream_t s, int *dev_status) {
    std::lock_guard<std::recursive_mutex> one_persistent_solve(persist_lock(R.device));
    Args<long long> a = resident_args(R);
    a.max_rounds = rounds > 0 ? R.r + rounds : 0;
    static int per_sm_cache[64] = {0};  // resident blocks per SM, per device
    int per_sm = R.device >= 0 && R.device < 64 ? per_sm_cache[R.device] : 0;
    if (per_sm < 1) {
        EG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fixpoint<true, long long>, THREADS, 0));
        if (per_sm < 1) {
            set_error("fixpoint kernel cannot be resident");
            return EG_ERR_CUDA;
        }
        if (R.device >= 0 && R.device < 64) per_sm_cache[R.device] = per_sm;
    }
    dim3 grid(num_sms(R.device) * per_sm), block(THREADS);
    void *args[] = {&a};
    EG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_fixpoint<true, long long>, grid, block, args, 0, s));
    EG_CUDA_TRY(cudaMemcpyAsync(R.host_ctrl, R.sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    const Ctrl *hc = (const Ctrl *)R.host_ctrl;
    *dev_status = hc->status;
    if (hc->status == DEV_OK) R.r = hc->r_next;
    return EG_OK;
}

eg_status resident_busy(Resident &R, cudaStream_t s) {
    EG_CUDA_TRY(cudaMemsetAsync(R.busy, 0, (size_t)R.slots * 4, s));
    const int r = (int)R.r;
    k_busy<<<num_sms(R.device) * 4, 256, 0, s>>>(R.sb.d.ctrl, r % 3, R.sb.d.pull_items[r & 1],
                                                 R.sb.d.push_items[r & 1], R.inst_id, R.busy);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemcpyAsync(R.host_busy, R.busy, (size_t)R.slots * 4, cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    return EG_OK;
}

}  // namespace eg

// ---------------------------------------------------------------------------
// Allocation-free single solve.
//
// Some callers cannot allocate device memory when they solve: a host program
// whose framework has already reserved the GPU's memory for its own caching
// allocator, or a latency-bound loop where a cudaMalloc / cudaFree would
// synchronise the device and stall every other stream.  For them the solver
// keeps its working memory (lists, dedupe bitmaps, partial minima, control
// block, the certified trials' bitmaps and the credits of their dual lifts)
// in one file-scope device array of fixed size, and it computes the credits
// straight in the caller's device output buffer.  Every GPU that loads the
// library holds this array until the process exits; every call reuses it.
// The solve takes the same route as eg_solve_credit (a first attempt with a
// short round budget, then certified trial caps), so it gives the same
// credits in about the same time.

namespace eg {

constexpr long long NOALLOC_MAX_N = EG_NOALLOC_MAX_VERTICES;
constexpr size_t NOALLOC_WORDS = (size_t)(NOALLOC_MAX_N + 31) / 32;
constexpr size_t noalloc_up(size_t x) { return (x + 255) & ~size_t(255); }
// layout: 8 lists of n ints, 7 bitmaps (5 of the solve state, the proven
// player-0 and player-1 vertices), n partial minima (int64), n counts, the
// int64 credits of the dual lifts, the cycle jumps' claim epochs (n ints),
// control block, counters (bound accumulators, trial counts, vertices
// jumped)
constexpr size_t NA_LISTS = 0;
constexpr size_t NA_BITS = NA_LISTS + 8 * noalloc_up((size_t)NOALLOC_MAX_N * 4);
constexpr size_t NA_ACC = NA_BITS + 7 * noalloc_up(NOALLOC_WORDS * 4);
constexpr size_t NA_DONE = NA_ACC + noalloc_up((size_t)NOALLOC_MAX_N * 8);
constexpr size_t NA_DUAL = NA_DONE + noalloc_up((size_t)NOALLOC_MAX_N * 4);
constexpr size_t NA_KCLAIM = NA_DUAL + noalloc_up((size_t)NOALLOC_MAX_N * 8);
constexpr size_t NA_CTRL = NA_KCLAIM + noalloc_up((size_t)NOALLOC_MAX_N * 4);
constexpr size_t NA_COUNT = NA_CTRL + noalloc_up(sizeof(Ctrl));
constexpr size_t NA_BYTES = NA_COUNT + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of g_noalloc_scratch, looked up (cudaGetSymbolAddress, with
// the device current) once per device and context: in host code the array's
// name is a host-side stand-in, never a device address.  The cache is keyed
// on the id of the current context, so a device reset or another context on
// the device gets a fresh lookup; where that id cannot be had, every call
// looks the address up.
struct ScratchAddr {
    unsigned long long ctx_id;
    void *addr;
};
static ScratchAddr g_noalloc_addr[64];
static std::mutex g_noalloc_mu;
// epoch counters of the claim array in g_noalloc_scratch, per device (the
// array starts zeroed when the library loads; 0 is never an epoch)
static unsigned g_noalloc_epoch[64];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if unknown); called under
// g_noalloc_mu.
static unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        resolved = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_cur, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_cur = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
    }
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static eg_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d out of range", device);
        return EG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long id = current_ctx_id();
    ScratchAddr &c = g_noalloc_addr[device];
    if (id == 0 || c.ctx_id != id || !c.addr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the solver scratch failed: %s", cudaGetErrorString(e));
            return EG_ERR_CUDA;
        }
        c.ctx_id = id;
        c.addr = p;
    }
    *out = (unsigned char *)c.addr;
    return EG_OK;
}

static eg_status solve_noalloc(eg_arena *ar, int credit_bits, long long scale, long long shift, void *out,
                               eg_stats *st, cudaStream_t s, long long max_rounds) {
    if (credit_bits != 32 && credit_bits != 64) {
        set_error("credit_bits must be 32 or 64 (credits are computed in the output buffer)");
        return EG_ERR_INVALID;
    }
    if (ar->n > NOALLOC_MAX_N) {
        set_error("arena has %d vertices; the allocation-free solve holds at most %lld", ar->n, NOALLOC_MAX_N);
        return EG_ERR_INVALID;
    }
    const long long sa = scale < 0 ? -scale : scale, sh = shift < 0 ? -shift : shift;
    if (sa > (1LL << 30) || sh > (1LL << 61)) {
        set_error("weight map out of range");
        return EG_ERR_INVALID;
    }
    int device = 0;
    EG_CUDA_TRY(cudaGetDevice(&device));
    if (device != ar->device) {
        set_error("the arena lives on device %d, the current device is %d", ar->device, device);
        return EG_ERR_INVALID;
    }
    // the kernels write credits straight through credits_out
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, out) != cudaSuccess ||
        (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        set_error("credits_out must be device memory (it holds the credits during the solve)");
        return EG_ERR_INVALID;
    }
    if (attr.type == cudaMemoryTypeDevice && attr.device != ar->device) {
        set_error("credits_out lives on device %d, the arena on device %d", attr.device, ar->device);
        return EG_ERR_INVALID;
    }
    if ((uintptr_t)out % (uintptr_t)(credit_bits / 8) != 0) {
        set_error("credits_out must be aligned to %d bytes", credit_bits / 8);
        return EG_ERR_INVALID;
    }
    unsigned char *base = nullptr;
    eg_status rc = noalloc_scratch(device, &base);
    if (rc != EG_OK) return rc;

    // bound C of the weight view, accumulated in the scratch
    unsigned long long *dcount = (unsigned long long *)(base + NA_COUNT);
    EG_CUDA_TRY(cudaMemsetAsync(dcount, 0, 16, s));
    k_bound<<<num_sms(device) * 8, 256, 0, s>>>(ar->d, WeightView{scale, shift, 0}, dcount, dcount + 1);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, dcount, 16, cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    const long long C = (long long)((unsigned long long *)ar->host_ctrl)[0];
    const long long wmax = (long long)((unsigned long long *)ar->host_ctrl)[1];
    if (credit_bits == 32 && C + wmax > 0x7fffffffLL - 1) {
        set_error("int32 credits cannot hold C + max|w'| = %lld", C + wmax);
        return EG_ERR_OVERFLOW;
    }
    if (scale == 1 && shift == 0) {
        ar->C_plain = C;
        ar->wmax_plain = wmax;
    }

    // the game's state laid over the scratch, with the output buffer as its
    // credit array; the dual lifts' state shares its lists, bitmaps, partial
    // minima and control block and has its own int64 credits
    const size_t n = (size_t)ar->n, words = (n + 31) / 32;
    StateBuffers sb, sd;
    sb.bits = credit_bits;
    sb.nf = ar->n;
    sb.dirty = true;
    sb.d.f = out;
    for (int k = 0; k < 2; ++k) {
        sb.d.pull_items[k] = (int *)(base + NA_LISTS + (4 * k + 0) * noalloc_up(n * 4));
        sb.d.pull_offs[k] = (int *)(base + NA_LISTS + (4 * k + 1) * noalloc_up(n * 4));
        sb.d.push_items[k] = (int *)(base + NA_LISTS + (4 * k + 2) * noalloc_up(n * 4));
        sb.d.push_offs[k] = (int *)(base + NA_LISTS + (4 * k + 3) * noalloc_up(n * 4));
        sb.d.bits_pull[k] = (unsigned *)(base + NA_BITS + k * noalloc_up(words * 4));
        sb.d.bits_push[k] = (unsigned *)(base + NA_BITS + (2 + k) * noalloc_up(words * 4));
    }
    sb.d.seed_bits = (unsigned *)(base + NA_BITS + 4 * noalloc_up(words * 4));
    sb.d.acc = base + NA_ACC;
    sb.d.acc_done = (int *)(base + NA_DONE);
    sb.d.ctrl = (Ctrl *)(base + NA_CTRL);
    sd = sb;
    sd.bits = 64;
    sd.d.f = base + NA_DUAL;

    SolveMem m;
    m.sb = &sb;
    m.sd = &sd;
    m.cert_w0 = (unsigned *)(base + NA_BITS + 5 * noalloc_up(words * 4));
    m.cert_w1 = (unsigned *)(base + NA_BITS + 6 * noalloc_up(words * 4));
    m.aux = dcount + 2;
    m.kick_claim = (unsigned *)(base + NA_KCLAIM);
    m.kick_epoch = &g_noalloc_epoch[device];
    m.kick_jumps = dcount + 4;
    m.fixed = true;
    m.in_place = true;
    return solve_route(ar, m, credit_bits, credit_bits, scale, shift, C, wmax, out, st, s, max_rounds);
}

}  // namespace eg

extern "C" eg_status eg_solve_credit_noalloc(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                                             void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds) {
    eg::clear_error();
    if (!arena || !credits_out) {
        eg::set_error("arena and credits_out are required");
        return EG_ERR_INVALID;
    }
    try {
        return eg::solve_noalloc(arena, credit_bits, w_scale, w_shift, credits_out, st, (cudaStream_t)cuda_stream,
                                 max_rounds);
    } catch (...) {
        eg::set_error("unexpected exception in eg_solve_credit_noalloc");
        return EG_ERR_INVALID;
    }
}
