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
    unsigned *bits[2];
    T *acc;
    int *acc_done;
    Ctrl *ctrl;
    long long max_rounds;
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
            for (int k = b; k < e; ++k) {
                T t = ominus<T>(T(0), wmap(__ldg(A.w + k), a.W), a.W.C);
                g = p1 ? max(g, t) : min(g, t);
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
    unsigned *bits = a.bits[r & 1];
    unsigned long long *push_ctr = &a.ctrl->push_ctr[r % 3];
    int *push_items = a.push_items[r & 1];
    int *push_offs = a.push_offs[r & 1];

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
        red[lane] = Cred<T>::TOP;
        __syncwarp();
        for (int xb = x; xb < stop; xb += 32) {
            const int xl = xb + lane;
            const bool act = xl < stop;
            int j = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                int oj = __shfl_sync(FULL, o, j + s);
                if (oj <= xl) j += s;
            }
            const int bj = __shfl_sync(FULL, beg, j);
            const int oj = __shfl_sync(FULL, o, j);
            T t = Cred<T>::TOP;
            if (act) {
                const int e = bj + (xl - oj);
                const int u = __ldg(A.col + e);
                t = ominus<T>(ld_cg(a.f + u), wmap(__ldg(A.w + e), a.W), a.W.C);
            }
            const int key = act ? j : 32 + lane;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                T ov = __shfl_up_sync(FULL, t, d);
                int ok = __shfl_up_sync(FULL, key, d);
                if (lane >= d && ok == key) t = min(t, ov);
            }
            const int nk = __shfl_down_sync(FULL, key, 1);
            if (act && (lane == 31 || nk != key)) red[j] = min(red[j], t);
            __syncwarp();
        }
        // finish the lifts of this window's entries
        const T g = red[lane];
        __syncwarp();
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
            if (done) {
                const T cur = ld_cg(a.f + v);
                if (res > cur) {
                    st_cg(a.f + v, res);
                    pwork = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
                    changed = pwork > 0;
                }
            }
        }
        warp_append(changed, (unsigned)v, pwork, push_ctr, push_items, push_offs);
        x = stop;
        i += 32;
    }
}

// ---------------------------------------------------------------------------
// Push phase: send the rises of the push list of round r to predecessors.
template <typename T>
__device__ void push_phase(const Args<T> &a, int r) {
    const DevArena &A = a.A;
    const int lane = lane_id();
    const unsigned long long ctr = ld_cg(&a.ctrl->push_ctr[r % 3]);
    const int cnt = (int)(ctr & 0xffffffffu);
    const int total = (int)(ctr >> 32);
    const int *items = a.push_items[r & 1];
    const int *offs = a.push_offs[r & 1];
    unsigned *bits_cur = a.bits[r & 1];
    unsigned *bits_next = a.bits[(r + 1) & 1];
    const int nx = (r + 1) % 3;
    unsigned long long *next_pull_ctr = &a.ctrl->pull_ctr[nx];
    unsigned long long *next_push_ctr = &a.ctrl->push_ctr[nx];
    int *next_pull_items = a.pull_items[(r + 1) & 1];
    int *next_pull_offs = a.pull_offs[(r + 1) & 1];
    int *next_push_items = a.push_items[(r + 1) & 1];
    int *next_push_offs = a.push_offs[(r + 1) & 1];

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
        int o = total, oend = total, beg = 0;
        T val = T(0);
        if (valid) {
            const unsigned raw = (unsigned)ld_cg(items + ii);
            const int v = (int)(raw & 0x7fffffffu);
            o = ld_cg(offs + ii);
            oend = ii + 1 < cnt ? ld_cg(offs + ii + 1) : total;
            beg = __ldg(A.rrow_ptr + v);
            val = ld_cg(a.f + v);
            if ((raw & P1_FLAG) && o >= lo && o < hi) atomicAnd(bits_cur + (v >> 5), ~(1u << (v & 31)));
        }
        const int stop = min(hi, __shfl_sync(FULL, oend, 31));
        for (int xb = x; xb < stop; xb += 32) {
            const int xl = xb + lane;
            const bool act = xl < stop;
            int j = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                int oj = __shfl_sync(FULL, o, j + s);
                if (oj <= xl) j += s;
            }
            const int bj = __shfl_sync(FULL, beg, j);
            const int oj = __shfl_sync(FULL, o, j);
            const T vj = __shfl_sync(FULL, val, j);
            bool want_pull = false, want_push = false;
            int p = 0, work = 0;
            if (act) {
                const int e = bj + (xl - oj);
                const unsigned pr = __ldg(A.rcol + e);
                p = (int)(pr & 0x7fffffffu);
                const T t = ominus<T>(vj, wmap(__ldg(A.rw + e), a.W), a.W.C);
                bool rose = false;
                if (pr & P1_FLAG) {
                    if (t > ld_cg(a.f + p)) rose = t > atomicMax(a.f + p, t);
                    if (rose) {
                        work = __ldg(A.rrow_ptr + p + 1) - __ldg(A.rrow_ptr + p);
                        rose = work > 0;
                    }
                } else {
                    rose = t > ld_cg(a.f + p);
                    if (rose) work = __ldg(A.row_ptr + p + 1) - __ldg(A.row_ptr + p);
                }
                if (rose) {
                    const unsigned bit = 1u << (p & 31);
                    unsigned *wd = bits_next + (p >> 5);
                    if (!(ld_cg(wd) & bit) && !(atomicOr(wd, bit) & bit)) {
                        want_push = (pr & P1_FLAG) != 0;
                        want_pull = !want_push;
                    }
                }
            }
            warp_append(want_pull, (unsigned)p, work, next_pull_ctr, next_pull_items, next_pull_offs);
            warp_append(want_push, (unsigned)p | P1_FLAG, work, next_push_ctr, next_push_items, next_push_offs);
        }
        x = stop;
        i += 32;
    }
}

// ---------------------------------------------------------------------------
// Persistent fixpoint kernel (Algorithm 3's while-loop on the device).
template <typename T>
__global__ void __launch_bounds__(THREADS) k_fixpoint(Args<T> a) {
    __shared__ T red_all[WARPS][32];
    T *red = red_all[threadIdx.x >> 5];
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
        push_phase<T>(a, r);
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
    size_t o_bits[2];
    for (int k = 0; k < 2; ++k) { o_bits[k] = off; off = align_up(off + words * 4); }
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
        sb.d.bits[k] = (unsigned *)(blk + o_bits[k]);
    }
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
        EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits[0], 0, ((size_t)n + 31) / 32 * 4, s));
        EG_CUDA_TRY(cudaMemsetAsync(sb.d.bits[1], 0, ((size_t)n + 31) / 32 * 4, s));
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
        a.bits[k] = sb.d.bits[k];
    }
    a.acc = (T *)sb.d.acc;
    a.acc_done = sb.d.acc_done;
    a.ctrl = sb.d.ctrl;
    a.max_rounds = max_rounds;

    EG_CUDA_TRY(cudaEventRecord(ar->ev0, s));
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
