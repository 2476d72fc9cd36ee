// Device helpers of the solver: credit encoding, the bounded (-) operator,
// coherent loads, warp-aggregated list appends and the grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eg_internal.h"

namespace eg {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned P1_FLAG = 0x80000000u;  // high bit of a list entry / reverse column
constexpr int THREADS = 256;               // threads per block of the persistent kernels
constexpr int WARPS = THREADS / 32;

// device status codes written into Ctrl::status
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_BUDGET = 2;

template <typename T> struct Cred;
template <> struct Cred<int> {
    static constexpr int TOP = 0x7fffffff;
};
template <> struct Cred<long long> {
    static constexpr long long TOP = 0x7fffffffffffffffLL;
};

// w' = scale * w - shift (the weight view of a threshold query)
__device__ __forceinline__ long long wmap(int w, const WeightView &v) { return v.scale * (long long)w - v.shift; }

// Extremes of w' = scale * w - shift over a vertex's out-edges, from the
// extremes of its raw weights (the map is monotone: increasing for
// scale >= 0, decreasing otherwise).
__device__ __forceinline__ long long wmap_min(int wmin, int wmax, const WeightView &v) {
    return v.scale >= 0 ? wmap(wmin, v) : wmap(wmax, v);
}
__device__ __forceinline__ long long wmap_max(int wmin, int wmax, const WeightView &v) {
    return v.scale >= 0 ? wmap(wmax, v) : wmap(wmin, v);
}

// a (-) b over {0..C} u {TOP} (Sec. 3.1, bounded by the codomain C_G):
// TOP stays TOP, a value above C becomes TOP, a negative one becomes 0.
template <typename T>
__device__ __forceinline__ T ominus(T a, long long b, long long C) {
    if (a == Cred<T>::TOP) return a;
    long long d = (long long)a - b;
    if (d > C) return Cred<T>::TOP;
    return d < 0 ? T(0) : T(d);
}

// Loads of data that other blocks write during the kernel: served from L2
// (the coherence point), never from a possibly stale L1 line.
__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ long long ld_cg(const long long *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ld_cg(const unsigned *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long *p) { return __ldcg(p); }

__device__ __forceinline__ void st_cg(int *p, int v) { __stcg(p, v); }
__device__ __forceinline__ void st_cg(long long *p, long long v) { __stcg(p, v); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bitmap updates that order the credit accesses around them: a vertex is
// marked queued with a release (after the rise that queued it) and unmarked
// with an acquire (before its credits are read), so a rise absorbed by an
// already-queued vertex is seen when that vertex is processed.
__device__ __forceinline__ unsigned atom_or_release(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.release.gpu.global.or.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned atom_and_acquire(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acquire.gpu.global.and.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Warp-aggregated append to a list with a packed counter (entries in the
// low 32 bits, total work in the high 32 bits).  Entry k of the list gets
// offs[k] = sum of the works of entries 0..k-1, so a list is its own
// exclusive scan.  Must be called by all 32 lanes (converged).
__device__ __forceinline__ void warp_append(bool want, unsigned item, int work, unsigned long long *ctr,
                                            int *items, int *offs) {
    unsigned mask = __ballot_sync(FULL, want);
    if (mask == 0) return;
    const int lane = lane_id();
    int wk = want ? work : 0;
    int incl = wk;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader)
        base = atomicAdd(ctr, ((unsigned long long)(unsigned)total << 32) | (unsigned long long)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    if (want) {
        unsigned idx = (unsigned)(base & 0xffffffffu) + __popc(mask & ((1u << lane) - 1u));
        items[idx] = (int)item;
        offs[idx] = (int)(base >> 32) + (incl - wk);
    }
}

// Largest i in [0, count) with offs[i] <= x, for a strictly increasing offs
// with offs[0] = 0 <= x.  32-ary search by the whole warp.
__device__ __forceinline__ int warp_find(const int *offs, int count, int x) {
    const int lane = lane_id();
    int lo = 0, hi = count;
    while (hi - lo > 32) {
        int step = (hi - lo + 31) >> 5;
        int idx = lo + lane * step;
        bool ok = idx < hi && ld_cg(offs + idx) <= x;
        unsigned b = __ballot_sync(FULL, ok);
        int k = 31 - __clz(b);
        int nlo = lo + k * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    int idx = lo + lane;
    bool ok = idx < hi && ld_cg(offs + idx) <= x;
    unsigned b = __ballot_sync(FULL, ok);
    return lo + (31 - __clz(b));
}

// Grid-wide barrier for a cooperatively launched grid.  Every wait has a
// wall-clock limit; on expiry the block records DEV_TIMEOUT and leaves.
// Returns false when the solve must stop (timeout or an earlier error).
__device__ __forceinline__ bool grid_barrier(Ctrl *c, unsigned nblocks, unsigned &gen,
                                             unsigned long long limit_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicExch(&c->bar_gen, gen + 1);
        } else {
            unsigned long long t0 = 0;
            unsigned spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if (++spins > 256) {
                    if (t0 == 0) t0 = global_ns();
                    if (global_ns() - t0 > limit_ns) {
                        atomicExch(&c->status, DEV_TIMEOUT);
                        break;
                    }
                    if (*(volatile int *)&c->status != DEV_OK) break;
                    __nanosleep(64);
                }
            }
        }
        gen += 1;
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)&c->status == DEV_OK;
}

}  // namespace eg
