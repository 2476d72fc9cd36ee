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
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

constexpr unsigned long long BARRIER_LIMIT_NS = 5000000000ull;  // 5 s per wait
constexpr int LOCAL_CAP = 256;  // entries of a warp's local worklist

__device__ __forceinline__ int xchg(int *p, int v) { return atomicExch(p, v); }
__device__ __forceinline__ long long xchg(long long *p, long long v) {
    return (long long)atomicExch((unsigned long long *)p, (unsigned long long)v);
}

template <typename T>
struct Args {
    DevArena A;
    WeightView W;
    T *f;
    int *pull_items[2];
    int *pull_offs[2];
    int *push_items[2];
    int *push_offs[2];
    unsigned *bits_pull[2];  // dedupe of the pull list of round parity k
    unsigned *bits_push[2];  // dedupe of the push list of round parity k
    const unsigned *seed_bits;  // warm start: vertices that start at TOP (or null)
    T *acc;
    int *acc_done;
    Ctrl *ctrl;
    long long max_rounds;
    int local_windows;  // per-warp budget of local windows per round (0: no chaining)
    int local_maxdeg;   // largest degree a vertex may have to be chained locally
};

// ---------------------------------------------------------------------------
// Bound C = M_G = sum_v max(0, max_e -w'(e)) and max |w'| (Sec. 3.1).
__global__ void k_bound(DevArena A, WeightView W, unsigned long long *out_C, unsigned long long *out_wmax) {
    long long sum = 0, wmax = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        int b = __ldg(A.row_ptr + v), e = __ldg(A.row_ptr + v + 1);
        long long worst = 0;
        for (int k = b; k < e; ++k) {
            long long wv = wmap(__ldg(A.w + k), W);
            worst = max(worst, -wv);
            wmax = max(wmax, wv < 0 ? -wv : wv);
        }
        sum += worst;
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
// Warm start.  A player-1 vertex u on a cycle of player-1 vertices whose
// weight (under the weight view) is negative is won by player 1: player 1
// can keep the play on that cycle forever, so every credit runs out
// (Lemma "EGcycles" with memoryless determinacy, Sec. 3).  Its least-EPM
// value is TOP, so starting it at TOP stays below the least fixpoint.
// Looked for: negative self-loops and 2-cycles u -> t -> u.  One warp per
// player-1 vertex compares each out-edge (u, t) with each in-edge (s, u)
// for s == t; vertices with out-degree x in-degree above max_pairs are
// skipped (the warm start is optional, missing a cycle only costs time).
__global__ void k_seed(DevArena A, WeightView W, long long max_pairs, unsigned *seed_bits,
                       unsigned long long *count) {
    const int lane = lane_id();
    const int nw = gridDim.x * (blockDim.x >> 5);
    unsigned found_total = 0;
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < A.n; u += nw) {
        if (!((__ldg(A.owner_bits + (u >> 5)) >> (u & 31)) & 1u)) continue;
        const int ob = __ldg(A.row_ptr + u), oe = __ldg(A.row_ptr + u + 1);
        const int ib = __ldg(A.rrow_ptr + u), ie = __ldg(A.rrow_ptr + u + 1);
        if ((long long)(oe - ob) * (long long)(ie - ib) > max_pairs) continue;
        bool found = false;
        for (int kb = ob; kb < oe; kb += 32) {
            const int k = kb + lane;
            int t = -1;
            long long wt = 0;
            if (k < oe) {
                t = __ldg(A.col + k);
                wt = wmap(__ldg(A.w + k), W);
                if (t == u && wt < 0) found = true;  // negative self-loop
            }
            for (int jb = ib; jb < ie; jb += 32) {
                const int j = jb + lane;
                unsigned sv = 0;
                long long ws = 0;
                if (j < ie) {
                    sv = __ldg(A.rcol + j);
                    ws = wmap(__ldg(A.rw + j), W);
                }
                const int cnt = min(32, ie - jb);
                for (int q = 0; q < cnt; ++q) {
                    const unsigned sq = __shfl_sync(FULL, sv, q);
                    const long long wq = __shfl_sync(FULL, ws, q);
                    if ((sq & P1_FLAG) && (int)(sq & 0x7fffffffu) == t && (int)(sq & 0x7fffffffu) != u &&
                        wt + wq < 0)
                        found = true;
                }
            }
        }
        if (__any_sync(FULL, found)) {
            if (lane == 0) atomicOr(seed_bits + (u >> 5), 1u << (u & 31));
            ++found_total;
        }
    }
    if (lane == 0 && found_total) atomicAdd(count, (unsigned long long)found_total);
}

// ---------------------------------------------------------------------------
// Initialisation (Algorithm 3, lines 1-3, with the first lift folded in):
// f(v) = delta(0, v)(v), i.e. max(0, -w') maximised (V1) or minimised (V0)
// over v's edges.  That is positive exactly for the initial set L of
// Algorithm 1 (V0 with every edge negative, V1 with some edge negative);
// those vertices enter push list 0.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_init(Args<T> a) {
    const DevArena &A = a.A;
    const int nthreads = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < A.n; base += nthreads) {
        int v = base + threadIdx.x;
        bool want = false;
        int work = 0;
        unsigned item = 0;
        if (v < A.n) {
            const bool p1 = (__ldg(A.owner_bits + (v >> 5)) >> (v & 31)) & 1u;
            const int b = __ldg(A.row_ptr + v), e = __ldg(A.row_ptr + v + 1);
            T g = p1 ? T(0) : Cred<T>::TOP;
            if (a.seed_bits && ((a.seed_bits[v >> 5] >> (v & 31)) & 1u)) {
                g = Cred<T>::TOP;
            } else {
                for (int k = b; k < e; ++k) {
                    T t = ominus<T>(T(0), wmap(__ldg(A.w + k), a.W), a.W.C);
                    g = p1 ? max(g, t) : min(g, t);
                }
            }
            a.f[v] = g;
            work = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
            want = g > T(0) && work > 0;
            item = (unsigned)v | (p1 ? P1_FLAG : 0u);
        }
        warp_append(want, item, work, &a.ctrl->push_ctr[0], a.push_items[0], a.push_offs[0]);
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
// owning lane (TOP for lanes that own none of them).
template <typename T>
__device__ __forceinline__ T pull_min(const Args<T> &a, int beg, int o, int x0, int stop, T *red) {
    const int lane = lane_id();
    red[lane] = Cred<T>::TOP;
    __syncwarp();
    for (int xb = x0; xb < stop; xb += 32) {
        const int xl = xb + lane;
        const bool act = xl < stop;
        const int j = owner_lane(o, xl);
        const int bj = __shfl_sync(FULL, beg, j);
        const int oj = __shfl_sync(FULL, o, j);
        T t = Cred<T>::TOP;
        if (act) {
            const int e = bj + (xl - oj);
            const int u = __ldg(a.A.col + e);
            t = ominus<T>(ld_cg(a.f + u), wmap(__ldg(a.A.w + e), a.W), a.W.C);
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

// Per-warp state of one round's push phase: the local worklist (a stack in
// shared memory) and counters of the work done through it.
template <typename T>
struct Local {
    int *stack;
    int top;
    bool on;
    unsigned long long relax, lifts, pushes;
};

constexpr unsigned NEED_NONE = 0, NEED_PULL = 1, NEED_PUSH = 2;

// Routes vertices that need work in this or the next round.  NEED_PULL: a
// player-0 vertex that may lift; NEED_PUSH: a vertex whose rise must reach
// its predecessors.  The next round's bitmap of that kind marks a vertex as
// queued -- in some warp's local worklist or in the next round's list -- so a
// vertex already queued absorbs the request (it reads fresh credits when it
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
    const int nx = (r + 1) % 3;
    warp_append(gpull, (unsigned)p, work, &a.ctrl->pull_ctr[nx], a.pull_items[(r + 1) & 1],
                a.pull_offs[(r + 1) & 1]);
    warp_append(gpush, (unsigned)p, work, &a.ctrl->push_ctr[nx], a.push_items[(r + 1) & 1],
                a.push_offs[(r + 1) & 1]);
}

// Sends the values `val` of the window's entries over their in-edges
// [x0, stop): t = val (-) w(p, v) for every predecessor p.  A player-1 p takes
// max(f(p), t) (atomicMax) and, if it rose, needs a push; a player-0 p with
// f(p) < t may need a lift.
template <typename T>
__device__ __forceinline__ void push_edges(const Args<T> &a, int r, int beg, int o, T val, int x0, int stop,
                                           Local<T> &L) {
    const int lane = lane_id();
    for (int xb = x0; xb < stop; xb += 32) {
        const int xl = xb + lane;
        const bool act = xl < stop;
        const int j = owner_lane(o, xl);
        const int bj = __shfl_sync(FULL, beg, j);
        const int oj = __shfl_sync(FULL, o, j);
        const T vj = __shfl_sync(FULL, val, j);
        unsigned need = NEED_NONE;
        int p = 0, work = 0;
        if (act) {
            const int e = bj + (xl - oj);
            const unsigned pr = __ldg(a.A.rcol + e);
            p = (int)(pr & 0x7fffffffu);
            const T t = ominus<T>(vj, wmap(__ldg(a.A.rw + e), a.W), a.W.C);
            if (t > ld_cg(a.f + p)) {
                if (pr & P1_FLAG) {
                    if (t > atomicMax(a.f + p, t)) {
                        work = __ldg(a.A.rrow_ptr + p + 1) - __ldg(a.A.rrow_ptr + p);
                        if (work > 0) need = NEED_PUSH;
                    }
                } else {
                    work = __ldg(a.A.row_ptr + p + 1) - __ldg(a.A.row_ptr + p);
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
template <typename T>
__device__ void drain_local(const Args<T> &a, int r, T *red, Local<T> &L) {
    const int lane = lane_id();
    int windows = 0;
    while (L.top > 0) {
        if (windows >= a.local_windows) L.on = false;
        ++windows;
        const int take = min(32, L.top);
        const bool have = lane < take;
        const int raw = have ? L.stack[L.top - 1 - lane] : 0;
        __syncwarp();
        L.top -= take;
        const int v = raw & 0x7fffffff;
        const bool is_push = have && (raw & (int)P1_FLAG);
        const bool is_pull = have && !(raw & (int)P1_FLAG);
        if (!L.on) {  // budget spent: the entries (still marked) join the next round's lists
            const int work = !have ? 0
                             : is_pull ? __ldg(a.A.row_ptr + v + 1) - __ldg(a.A.row_ptr + v)
                                       : __ldg(a.A.rrow_ptr + v + 1) - __ldg(a.A.rrow_ptr + v);
            const int nx = (r + 1) % 3;
            warp_append(is_pull, (unsigned)v, work, &a.ctrl->pull_ctr[nx], a.pull_items[(r + 1) & 1],
                        a.pull_offs[(r + 1) & 1]);
            warp_append(is_push, (unsigned)v, work, &a.ctrl->push_ctr[nx], a.push_items[(r + 1) & 1],
                        a.push_offs[(r + 1) & 1]);
            continue;
        }
        if (have) {  // unmark before reading credits
            unsigned *bits = is_pull ? a.bits_pull[(r + 1) & 1] : a.bits_push[(r + 1) & 1];
            atom_and_acquire(bits + (v >> 5), ~(1u << (v & 31)));
        }
        // lifts
        int pbeg = 0, pwork = 0;
        if (is_pull) {
            pbeg = __ldg(a.A.row_ptr + v);
            pwork = __ldg(a.A.row_ptr + v + 1) - pbeg;
        }
        int po;
        const int ptotal = warp_exclusive(pwork, po);
        T g = Cred<T>::TOP;
        if (ptotal > 0) g = pull_min<T>(a, pbeg, po, 0, ptotal, red);
        bool rose = is_push;
        T val = T(0);
        if (is_pull) {
            rose = g > atomicMax(a.f + v, g);
            val = g;
        } else if (is_push) {
            val = ld_cg(a.f + v);
        }
        L.relax += ptotal;
        L.lifts += __popc(__ballot_sync(FULL, is_pull));
        // pushes: small ones here, large ones to the next round
        int qbeg = 0, qwork = 0;
        if (rose) {
            qbeg = __ldg(a.A.rrow_ptr + v);
            qwork = __ldg(a.A.rrow_ptr + v + 1) - qbeg;
        }
        const bool big = rose && qwork > a.local_maxdeg;
        {
            bool gpush = false;
            if (big) {
                const unsigned bit = 1u << (v & 31);
                gpush = !(atom_or_release(a.bits_push[(r + 1) & 1] + (v >> 5), bit) & bit);
            }
            warp_append(gpush, (unsigned)v, qwork, &a.ctrl->push_ctr[(r + 1) % 3], a.push_items[(r + 1) & 1],
                        a.push_offs[(r + 1) & 1]);
        }
        if (big || !rose) qwork = 0;
        int qo;
        const int qtotal = warp_exclusive(qwork, qo);
        if (qtotal > 0) push_edges<T>(a, r, qbeg, qo, val, 0, qtotal, L);
        L.relax += qtotal;
        L.pushes += __popc(__ballot_sync(FULL, qwork > 0));
    }
}

// ---------------------------------------------------------------------------
// Pull phase: lift the player-0 vertices of the pull list of round r.
template <typename T>
__device__ void pull_phase(const Args<T> &a, int r, T *red) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const unsigned long long ctr = ld_cg(&a.ctrl->pull_ctr[r % 3]);
    const int cnt = (int)(ctr & 0xffffffffu);
    const int total = (int)(ctr >> 32);
    const int *items = a.pull_items[r & 1];
    const int *offs = a.pull_offs[r & 1];
    unsigned *bits = a.bits_pull[r & 1];
    unsigned *bits_q = a.bits_push[r & 1];

    const int nwarps = gridDim.x * WARPS;
    const int gw = blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int K = max(32, (total + nwarps - 1) / nwarps);
    const int lo = gw * K;
    if (lo >= total) return;
    const int hi = min(total, lo + K);

    int i = warp_find(offs, cnt, lo);
    int x = lo;
    while (x < hi) {
        const int ii = i + lane;
        const bool valid = ii < cnt;
        int v = 0, o = total, oend = total, beg = 0;
        if (valid) {
            v = ld_cg(items + ii) & 0x7fffffff;
            o = ld_cg(offs + ii);
            oend = ii + 1 < cnt ? ld_cg(offs + ii + 1) : total;
            beg = __ldg(A.row_ptr + v);
        }
        const int stop = min(hi, __shfl_sync(FULL, oend, 31));
        const T g = pull_min<T>(a, beg, o, x, stop, red);
        // finish the lifts of this window's entries
        bool changed = false;
        int pwork = 0;
        if (valid && o < stop && oend > x) {
            if (o >= lo) atomicAnd(bits + (v >> 5), ~(1u << (v & 31)));  // consumed
            const int seen = min(oend, stop) - max(o, x);
            T res = g;
            bool done = true;
            if (seen != oend - o) {  // lift split across warps: merge partial minima
                atomicMin(a.acc + v, g);
                __threadfence();
                const int before = atomicAdd(a.acc_done + v, seen);
                done = before + seen == oend - o;
                if (done) {
                    __threadfence();
                    res = xchg(a.acc + v, Cred<T>::TOP);
                    atomicExch(a.acc_done + v, 0);
                }
            }
            if (done && res > ld_cg(a.f + v) && res > atomicMax(a.f + v, res)) {
                pwork = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
                if (pwork > 0) {
                    const unsigned bit = 1u << (v & 31);
                    changed = !(ld_cg(bits_q + (v >> 5)) & bit) && !(atomicOr(bits_q + (v >> 5), bit) & bit);
                }
            }
        }
        warp_append(changed, (unsigned)v, pwork, &a.ctrl->push_ctr[r % 3], a.push_items[r & 1],
                    a.push_offs[r & 1]);
        x = stop;
        i += 32;
    }
}

// ---------------------------------------------------------------------------
// Push phase: send the rises of the push list of round r to predecessors,
// then work through the warp's local worklist.
template <typename T>
__device__ void push_phase(const Args<T> &a, int r, T *red, Local<T> &L) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const unsigned long long ctr = ld_cg(&a.ctrl->push_ctr[r % 3]);
    const int cnt = (int)(ctr & 0xffffffffu);
    const int total = (int)(ctr >> 32);
    const int *items = a.push_items[r & 1];
    const int *offs = a.push_offs[r & 1];
    unsigned *bits_cur = a.bits_push[r & 1];

    const int nwarps = gridDim.x * WARPS;
    const int gw = blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int K = max(32, (total + nwarps - 1) / nwarps);
    const int lo = gw * K;
    L.top = 0;
    L.on = a.local_windows > 0;
    if (lo >= total) return;
    const int hi = min(total, lo + K);

    int i = warp_find(offs, cnt, lo);
    int x = lo;
    while (x < hi) {
        const int ii = i + lane;
        const bool valid = ii < cnt;
        int o = total, oend = total, beg = 0;
        T val = T(0);
        if (valid) {
            const int v = ld_cg(items + ii) & 0x7fffffff;
            o = ld_cg(offs + ii);
            oend = ii + 1 < cnt ? ld_cg(offs + ii + 1) : total;
            beg = __ldg(A.rrow_ptr + v);
            if (o >= lo && o < hi) atomicAnd(bits_cur + (v >> 5), ~(1u << (v & 31)));  // consumed
            val = ld_cg(a.f + v);
        }
        const int stop = min(hi, __shfl_sync(FULL, oend, 31));
        push_edges<T>(a, r, beg, o, val, x, stop, L);
        x = stop;
        i += 32;
    }
    drain_local<T>(a, r, red, L);
}

// ---------------------------------------------------------------------------
// Persistent fixpoint kernel (Algorithm 3's while-loop on the device).
template <typename T>
__global__ void __launch_bounds__(THREADS) k_fixpoint(Args<T> a) {
    __shared__ T red_all[WARPS][32];
    __shared__ int stack_all[WARPS][LOCAL_CAP];
    const int wid = threadIdx.x >> 5;
    T *red = red_all[wid];
    Local<T> L;
    L.stack = stack_all[wid];
    L.top = 0;
    L.on = false;
    L.relax = L.lifts = L.pushes = 0;
    Ctrl *c = a.ctrl;
    unsigned gen = 0;
    for (int r = 0;; ++r) {
        if (a.max_rounds > 0 && r >= a.max_rounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&c->status, DEV_BUDGET);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->pull_ctr[(r + 2) % 3] = 0;
            c->push_ctr[(r + 2) % 3] = 0;
        }
        const unsigned long long pc = ld_cg(&c->pull_ctr[r % 3]);
        if ((pc & 0xffffffffu) != 0) {
            pull_phase<T>(a, r, red);
            if (!grid_barrier(c, gridDim.x, gen, BARRIER_LIMIT_NS)) break;
        }
        const unsigned long long qc = ld_cg(&c->push_ctr[r % 3]);
        push_phase<T>(a, r, red, L);
        if (!grid_barrier(c, gridDim.x, gen, BARRIER_LIMIT_NS)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->rounds += 1;
            c->lifts += pc & 0xffffffffu;
            c->pushes += qc & 0xffffffffu;
            c->relax += (pc >> 32) + (qc >> 32);
        }
        const unsigned long long np = ld_cg(&c->pull_ctr[(r + 1) % 3]);
        const unsigned long long nq = ld_cg(&c->push_ctr[(r + 1) % 3]);
        if (blockIdx.x == 0 && threadIdx.x == 0) c->enqueues += (np & 0xffffffffu) + (nq & 0xffffffffu);
        if ((np & 0xffffffffu) == 0 && (nq & 0xffffffffu) == 0) break;
    }
    if (lane_id() == 0 && (L.relax | L.lifts | L.pushes)) {
        atomicAdd(&c->relax, L.relax);
        atomicAdd(&c->lifts, L.lifts);
        atomicAdd(&c->pushes, L.pushes);
    }
}

// ---------------------------------------------------------------------------
// Host side

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

static eg_status ensure_state(eg_arena *ar, int bits) {
    StateBuffers &sb = bits == 32 ? ar->st32 : ar->st64;
    if (sb.bits == bits) return EG_OK;
    const size_t n = (size_t)ar->n, cs = bits / 8, words = (n + 31) / 32;
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

template <typename T>
static eg_status launch_solve(eg_arena *ar, StateBuffers &sb, const WeightView &W, cudaStream_t s,
                              long long max_rounds) {
    const int n = ar->n;
    const int sms = num_sms(ar->device);
    if (sb.dirty) {
        k_fill<T><<<sms * 4, 256, 0, s>>>((T *)sb.d.acc, n, Cred<T>::TOP);
        EG_CUDA_TRY(cudaMemsetAsync(sb.d.acc_done, 0, (size_t)n * 4, s));
        for (int k = 0; k < 2; ++k) {
            EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits_pull[k], 0, ((size_t)n + 31) / 32 * 4, s));
            EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits_push[k], 0, ((size_t)n + 31) / 32 * 4, s));
        }
        sb.dirty = false;
    }
    EG_CUDA_TRY(cudaMemsetAsync(sb.d.ctrl, 0, sizeof(Ctrl), s));
    Args<T> a;
    a.A = ar->d;
    a.W = W;
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
    a.max_rounds = max_rounds;
    a.local_windows = ar->local_windows;
    a.local_maxdeg = ar->local_maxdeg;

    EG_CUDA_TRY(cudaEventRecord(ar->ev0, s));
    a.seed_bits = nullptr;
    if (ar->warm_start) {
        EG_CUDA_TRY(cudaMemsetAsync(sb.d.seed_bits, 0, ((size_t)n + 31) / 32 * 4, s));
        const int sblocks = (int)std::min<long long>(((long long)n + 7) / 8, (long long)sms * 32);
        k_seed<<<sblocks, 256, 0, s>>>(ar->d, W, ar->seed_max_pairs, sb.d.seed_bits, &sb.d.ctrl->seeded);
        EG_CUDA_TRY(cudaGetLastError());
        a.seed_bits = sb.d.seed_bits;
    }
    const int init_blocks = (int)std::min<long long>((n + THREADS - 1) / THREADS, (long long)sms * 16);
    k_init<T><<<init_blocks, THREADS, 0, s>>>(a);
    EG_CUDA_TRY(cudaGetLastError());

    int per_sm = 0;
    EG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fixpoint<T>, THREADS, 0));
    if (per_sm < 1) {
        set_error("fixpoint kernel cannot be resident");
        return EG_ERR_CUDA;
    }
    dim3 grid(sms * per_sm), block(THREADS);
    void *args[] = {&a};
    EG_CUDA_TRY(cudaEventRecord(ar->evk, s));
    EG_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_fixpoint<T>, grid, block, args, 0, s));
    EG_CUDA_TRY(cudaEventRecord(ar->ev1, s));
    return EG_OK;
}

__global__ void k_widen(const int *in, long long *out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int v = in[i];
        out[i] = v == Cred<int>::TOP ? Cred<long long>::TOP : (long long)v;
    }
}

eg_status solve(eg_arena *ar, int credit_bits, long long scale, long long shift, void *out, eg_stats *st,
                cudaStream_t s, long long max_rounds) {
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
    StateBuffers &sb = bits == 32 ? ar->st32 : ar->st64;
    WeightView W{scale, shift, C};
    rc = bits == 32 ? launch_solve<int>(ar, sb, W, s, max_rounds) : launch_solve<long long>(ar, sb, W, s, max_rounds);
    if (rc != EG_OK) return rc;

    // credits out: same width, or widened to int64 when credit_bits == 0
    const int out_bits = credit_bits == 0 ? 64 : bits;
    cudaPointerAttributes attr{};
    bool dev_out = cudaPointerGetAttributes(&attr, out) == cudaSuccess &&
                   (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    void *src = sb.d.f;
    void *tmp = nullptr;
    if (out_bits != bits) {  // widen int32 -> int64 with TOP mapped
        EG_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)ar->n * 8, s));
        const int wb = std::min((ar->n + 255) / 256, 4096);
        k_widen<<<wb, 256, 0, s>>>((const int *)sb.d.f, (long long *)tmp, ar->n);
        EG_CUDA_TRY(cudaGetLastError());
        src = tmp;
    }
    EG_CUDA_TRY(cudaMemcpyAsync(out, src, (size_t)ar->n * (out_bits / 8),
                                dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (tmp) EG_CUDA_TRY(cudaFreeAsync(tmp, s));
    EG_CUDA_TRY(cudaMemcpyAsync(ar->host_ctrl, sb.d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    const Ctrl *hc = (const Ctrl *)ar->host_ctrl;
    float ms = 0.f, kms = 0.f;
    cudaEventElapsedTime(&ms, ar->ev0, ar->ev1);
    cudaEventElapsedTime(&kms, ar->evk, ar->ev1);
    eg_status result = EG_OK;
    if (hc->status == DEV_TIMEOUT) {
        set_error("a device-side wait exceeded its limit");
        result = EG_ERR_TIMEOUT;
        sb.dirty = true;
    } else if (hc->status == DEV_BUDGET) {
        set_error("round budget of %lld exhausted", max_rounds);
        result = EG_ERR_BUDGET;
        sb.dirty = true;
    }
    if (st) {
        st->C = C;
        st->seeded = (int64_t)hc->seeded;
        st->credit_bits = bits;
        st->status = result;
        st->rounds = (int64_t)hc->rounds;
        st->lifts = (int64_t)hc->lifts;
        st->pushes = (int64_t)hc->pushes;
        st->relaxations = (int64_t)hc->relax;
        st->enqueues = (int64_t)hc->enqueues;
        st->ms = ms;
        st->fixpoint_ms = kms;
    }
    return result;
}

}  // namespace eg
