// Arena construction and the C ABI entry points of libeg.
//
// eg_create copies the forward CSR of the arena (Sec. 2) to the device,
// validates it there (offsets, ids, totality), narrows the offsets to int32
// and builds the predecessor sets pre(v) (Sec. 2) as a reverse CSR with the
// owner of each predecessor in the high bit of its id: the paper's redundant
// CSC representation (Sec. 5), built here by our own count / scan / scatter
// kernels rather than a library transpose.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

enum : unsigned { BAD_ROWPTR = 1u, NOT_TOTAL = 2u, BAD_COL = 4u, BAD_RROWPTR = 8u, BAD_RCOL = 16u };

// Validates the int64 forward offsets and narrows them to int32.
__global__ void k_check_rows(const long long *rp64, int n, int m, int *rp32, unsigned *flags) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        long long a = rp64[v];
        unsigned f = 0;
        if (a < 0 || a > m) f |= BAD_ROWPTR;
        if (v == 0 && a != 0) f |= BAD_ROWPTR;
        if (v == n && a != m) f |= BAD_ROWPTR;
        if (v < n) {
            long long b = rp64[v + 1];
            if (b < a) f |= BAD_ROWPTR;
            else if (b == a) f |= NOT_TOTAL;
        }
        rp32[v] = (int)a;
        if (f) atomicOr(flags, f);
    }
}

__global__ void k_check_cols(const int *col, int m, int n, unsigned *flags, unsigned bad) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        unsigned c = (unsigned)col[e] & (bad == BAD_RCOL ? 0x7fffffffu : 0xffffffffu);
        if (c >= (unsigned)n) atomicOr(flags, bad);
    }
}

// in-degree counts into cnt[0..n-1] (cnt zeroed by the caller)
__global__ void k_fill_int(int *p, int n, int v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_count_in(const int *col, int m, int *cnt) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
        atomicAdd(cnt + col[e], 1);
}

// Block-local exclusive scan of data[0..len) in place; block totals to sums.
__global__ void k_scan_blocks(int *data, int len, int *sums) {
    __shared__ int warp_tot[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = i < len ? data[i] : 0;
    int incl = x;
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int ti = t;
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(FULL, ti, d);
            if (lane >= d) ti += o;
        }
        warp_tot[lane] = ti - t;
        if (lane == 31 && sums) sums[blockIdx.x] = ti;
    }
    __syncthreads();
    if (i < len) data[i] = incl - x + warp_tot[wid];
}

__global__ void k_add_offsets(int *data, int len, const int *offs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) data[i] += offs[blockIdx.x];
}

// Exclusive scan of data[0..len) in place; scratch holds the block sums of
// every level (at most len / 1024 + 64 ints).
static cudaError_t exclusive_scan(int *data, int len, int *scratch, cudaStream_t s) {
    const int B = 1024;
    int nb = (len + B - 1) / B;
    if (nb <= 1) {
        k_scan_blocks<<<1, B, 0, s>>>(data, len, nullptr);
        return cudaGetLastError();
    }
    k_scan_blocks<<<nb, B, 0, s>>>(data, len, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan(scratch, nb, scratch + nb, s);
    if (e != cudaSuccess) return e;
    k_add_offsets<<<nb, B, 0, s>>>(data, len, scratch);
    return cudaGetLastError();
}

// Row work is split by degree so that hubs do not serialise: a row of at
// most TIER0 edges goes to one thread; longer rows are collected into
// grid-wide lists, a row of at most TIER1 edges to one warp, a longer one to
// a whole block (k_collect_rows, for_long_rows).
constexpr int TIER0 = 16;
constexpr int TIER1 = 2048;

__device__ __forceinline__ int row_tier(int deg) { return deg <= TIER0 ? 0 : (deg <= TIER1 ? 1 : 2); }

// Scatter of one out-edge k of row v into the reverse CSR.
__device__ __forceinline__ void scatter_edge(int k, unsigned tag, const int *col, const int *w, int *fill,
                                             unsigned *rcol, int *rw) {
    const int slot = atomicAdd(fill + col[k], 1);
    rcol[slot] = tag;
    rw[slot] = w[k];
}

__device__ __forceinline__ unsigned owner_tag(const unsigned *owner_bits, int v) {
    return (unsigned)v | ((((owner_bits[v >> 5] >> (v & 31)) & 1u) != 0) ? P1_FLAG : 0u);
}

// Scatter of the short rows (at most TIER0 edges) into the reverse CSR: one
// thread per row, all of its cursor atomics in flight at once.  Longer rows
// go through k_collect_rows / k_scatter_long.
__global__ void k_scatter(int n, const int *row_ptr, const int *col, const int *w, const unsigned *owner_bits,
                          int *fill, unsigned *rcol, int *rw) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int b = row_ptr[v], deg = row_ptr[v + 1] - b;
        if (row_tier(deg) != 0) continue;
        const unsigned tag = owner_tag(owner_bits, v);
        int dst[TIER0], wt[TIER0], slot[TIER0];
#pragma unroll
        for (int k = 0; k < TIER0; ++k)
            if (k < deg) {
                dst[k] = col[b + k];
                wt[k] = w[b + k];
            }
#pragma unroll
        for (int k = 0; k < TIER0; ++k)
            if (k < deg) slot[k] = atomicAdd(fill + dst[k], 1);
#pragma unroll
        for (int k = 0; k < TIER0; ++k)
            if (k < deg) {
                rcol[slot[k]] = tag;
                rw[slot[k]] = wt[k];
            }
    }
}

// Smallest and largest weight of every short row (rows are never empty
// here): one thread per row, its loads all in flight at once.  Longer rows go
// through k_row_extremes_long.
__global__ void k_row_extremes(int n, const int *row_ptr, const int *w, int *wmin, int *wmax) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int b = row_ptr[v], deg = row_ptr[v + 1] - b;
        if (row_tier(deg) != 0) continue;
        int lo = 0x7fffffff, hi = (int)0x80000000;
#pragma unroll
        for (int k = 0; k < TIER0; ++k)
            if (k < deg) {
                const int x = w[b + k];
                lo = min(lo, x);
                hi = max(hi, x);
            }
        wmin[v] = lo;
        wmax[v] = hi;
    }
}

// Rows longer than TIER0 edges, collected into two global lists (tier 1:
// up to TIER1 edges, tier 2: longer), so that their work spreads over the
// whole grid: R-MAT hubs sit at small vertex ids, and a per-chunk split
// would leave them to a few blocks.
__global__ void k_collect_rows(int n, const int *row_ptr, int *list1, int *cnt1, int *list2, int *cnt2) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int t = row_tier(row_ptr[v + 1] - row_ptr[v]);
        if (t == 1) list1[atomicAdd(cnt1, 1)] = v;
        else if (t == 2) list2[atomicAdd(cnt2, 1)] = v;
    }
}

// fn(v, begin, end, first, step) over the collected long rows: a tier-1 row
// to one warp of the grid, a tier-2 row to one block, both round robin.
template <typename F>
__device__ __forceinline__ void for_long_rows(const int *row_ptr, const int *list1, const int *cnt1,
                                              const int *list2, const int *cnt2, F fn) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int c1 = *cnt1, c2 = *cnt2;
    for (int k = gwarp; k < c1; k += nwarps) {
        const int v = list1[k];
        fn(v, row_ptr[v], row_ptr[v + 1], lane, 32);
    }
    for (int k = blockIdx.x; k < c2; k += gridDim.x) {
        const int v = list2[k];
        fn(v, row_ptr[v], row_ptr[v + 1], (int)threadIdx.x, (int)blockDim.x);
    }
}

__global__ void k_scatter_long(const int *row_ptr, const int *col, const int *w, const unsigned *owner_bits,
                               const int *list1, const int *cnt1, const int *list2, const int *cnt2, int *fill,
                               unsigned *rcol, int *rw) {
    for_long_rows(row_ptr, list1, cnt1, list2, cnt2, [&](int v, int b, int e, int first, int step) {
        const unsigned tag = owner_tag(owner_bits, v);
        for (int k = b + first; k < e; k += step) scatter_edge(k, tag, col, w, fill, rcol, rw);
    });
}

// Weight extremes of the long rows; wmin / wmax start at (INT_MAX, INT_MIN).
__global__ void k_row_extremes_long(const int *row_ptr, const int *w, const int *list1, const int *cnt1,
                                    const int *list2, const int *cnt2, int *wmin, int *wmax) {
    for_long_rows(row_ptr, list1, cnt1, list2, cnt2, [&](int v, int b, int e, int first, int step) {
        int lo = 0x7fffffff, hi = (int)0x80000000;
        for (int k = b + first; k < e; k += step) {
            lo = min(lo, w[k]);
            hi = max(hi, w[k]);
        }
        for (int d = 16; d; d >>= 1) {
            lo = min(lo, __shfl_xor_sync(FULL, lo, d));
            hi = max(hi, __shfl_xor_sync(FULL, hi, d));
        }
        if ((threadIdx.x & 31) == 0 && lo <= hi) {  // the warp saw an edge of the row
            atomicMin(wmin + v, lo);
            atomicMax(wmax + v, hi);
        }
    });
}

// Tags caller-provided reverse columns with the owner bit of the predecessor.
__global__ void k_tag_rcol(int m, const unsigned *owner_bits, unsigned *rcol) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        unsigned p = rcol[e] & 0x7fffffffu;
        rcol[e] = p | ((((owner_bits[p >> 5] >> (p & 31)) & 1u) != 0) ? P1_FLAG : 0u);
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long edge_hash(unsigned src, unsigned dst, int w) {
    return mix64(((unsigned long long)src << 32 | dst) ^ mix64(0x9E3779B97F4A7C15ull + (unsigned)w));
}

// Multiset hash of the forward edges (sum of per-edge hashes), one warp per row.
__global__ void k_hash_fwd(int n, const int *row_ptr, const int *col, const int *w, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    unsigned long long h = 0;
    for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
        const int b = row_ptr[v], e = row_ptr[v + 1];
        for (int k = b + lane; k < e; k += 32) h += edge_hash((unsigned)v, (unsigned)col[k], w[k]);
    }
    for (int d = 16; d; d >>= 1) h += __shfl_down_sync(FULL, h, d);
    if (lane == 0) atomicAdd(out, h);
}

__global__ void k_hash_rev(int n, const int *rrow_ptr, const unsigned *rcol, const int *rw, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    unsigned long long h = 0;
    for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
        const int b = rrow_ptr[v], e = rrow_ptr[v + 1];
        for (int k = b + lane; k < e; k += 32) h += edge_hash(rcol[k] & 0x7fffffffu, (unsigned)v, rw[k]);
    }
    for (int d = 16; d; d >>= 1) h += __shfl_down_sync(FULL, h, d);
    if (lane == 0) atomicAdd(out, h);
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

static int num_sms_arena(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms > 0 ? sms : 1;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes attr{};
    bool dev = p && cudaPointerGetAttributes(&attr, p) == cudaSuccess &&
               (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev;
}

static eg_status destroy(eg_arena *a) {
    if (!a) return EG_OK;
    free_state(a->st32);
    free_state(a->st64);
    free_state(a->st_dual);
    free_state(a->st_dual32);
    if (a->scc_level) cudaFree(a->scc_level);
    if (a->scc_comp) cudaFree(a->scc_comp);
    if (a->block) cudaFree(a->block);
    if (a->cert_block) cudaFree(a->cert_block);
    if (a->kick_block) cudaFree(a->kick_block);
    if (a->ev0) cudaEventDestroy(a->ev0);
    if (a->ev1) cudaEventDestroy(a->ev1);
    if (a->evk) cudaEventDestroy(a->evk);
    if (a->host_ctrl) cudaFreeHost(a->host_ctrl);
    delete a;
    return EG_OK;
}

static eg_status create(int64_t n64, int64_t m64, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                        const int64_t *rrow_ptr, const int32_t *rcol, const int32_t *rw,
                        const uint32_t *owner_bits, uint32_t flags, eg_arena **out) {
    if (!out) {
        set_error("out is NULL");
        return EG_ERR_INVALID;
    }
    *out = nullptr;
    if (n64 < 1 || n64 >= (1LL << 31) - 1 || m64 < n64 || m64 >= (1LL << 31) - 1) {
        set_error("need 1 <= n < 2^31 - 1 and n <= m < 2^31 - 1 (got n=%lld m=%lld)", (long long)n64,
                  (long long)m64);
        return m64 < n64 && n64 >= 1 && m64 >= 0 ? EG_ERR_NOT_TOTAL : EG_ERR_INVALID;
    }
    if (!row_ptr || !col || !w || !owner_bits) {
        set_error("row_ptr, col, w and owner_bits are required");
        return EG_ERR_INVALID;
    }
    const bool have_rev = rrow_ptr || rcol || rw;
    if (have_rev && !(rrow_ptr && rcol && rw)) {
        set_error("rrow_ptr, rcol and rw must be given together or all NULL");
        return EG_ERR_INVALID;
    }
    if ((flags & ~EG_INPUT_DEVICE) != 0) {
        set_error("unknown flags 0x%x", flags);
        return EG_ERR_INVALID;
    }
    const bool dev_in = (flags & EG_INPUT_DEVICE) != 0;
    if (dev_in && !is_device_ptr(row_ptr)) {
        set_error("EG_INPUT_DEVICE given but row_ptr is not device memory");
        return EG_ERR_INVALID;
    }
    const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int n = (int)n64, m = (int)m64;
    const size_t words = ((size_t)n + 31) / 32;

    eg_arena *a = new (std::nothrow) eg_arena();
    if (!a) {
        set_error("host allocation failed");
        return EG_ERR_OOM;
    }
    cudaGetDevice(&a->device);
    a->n = n;
    a->m = m;
    // EG_OPT_CERTIFY_AFTER's default: 8 plain rounds finish the games that
    // need no trials (R-MAT, most threshold queries) and hand the others to
    // the certified trials early; the results do not depend on it
    a->certify_after = 8;
    eg_status rc = EG_OK;
    char *tmp = nullptr;
#define TRY(expr)                     \
    do {                              \
        cudaError_t _e = (expr);      \
        if (_e != cudaSuccess) {      \
            set_error("%s failed: %s", #expr, cudaGetErrorString(_e)); \
            rc = _e == cudaErrorMemoryAllocation ? EG_ERR_OOM : EG_ERR_CUDA; \
            goto fail;                \
        }                             \
    } while (0)
    {
        // persistent arrays
        size_t off = 0;
        const size_t o_rp = off; off = align_up(off + ((size_t)n + 1) * 4);
        const size_t o_col = off; off = align_up(off + (size_t)m * 4);
        const size_t o_w = off; off = align_up(off + (size_t)m * 4);
        const size_t o_rrp = off; off = align_up(off + ((size_t)n + 1) * 4);
        const size_t o_rcol = off; off = align_up(off + (size_t)m * 4);
        const size_t o_rw = off; off = align_up(off + (size_t)m * 4);
        const size_t o_own = off; off = align_up(off + words * 4);
        const size_t o_wmin = off; off = align_up(off + (size_t)n * 4);
        const size_t o_wmax = off; off = align_up(off + (size_t)n * 4);
        char *blk = nullptr;
        unsigned *hflags = nullptr;
        unsigned long long hh[2] = {0, 0};
        const cudaStream_t s = 0;
        TRY(cudaMalloc((void **)&blk, off));
        a->block = blk;
        int *rp32 = (int *)(blk + o_rp);
        int *dcol = (int *)(blk + o_col);
        int *dw = (int *)(blk + o_w);
        int *rrp32 = (int *)(blk + o_rrp);
        unsigned *drcol = (unsigned *)(blk + o_rcol);
        int *drw = (int *)(blk + o_rw);
        unsigned *down = (unsigned *)(blk + o_own);
        int *dwmin = (int *)(blk + o_wmin);
        int *dwmax = (int *)(blk + o_wmax);
        // temporaries: int64 offsets (x2), flags, hashes, scan scratch, fill pointers
        size_t t = 0;
        const size_t t_rp = t; t = align_up(t + ((size_t)n + 1) * 8);
        const size_t t_rrp = t; t = align_up(t + ((size_t)n + 1) * 8);
        const size_t t_flags = t; t = align_up(t + 64);
        const size_t t_scan = t; t = align_up(t + ((size_t)n / 1024 + 64) * 4 * 2);
        const size_t t_fill = t; t = align_up(t + ((size_t)n + 1) * 4);
        // long-row lists: tier 1 (at most n rows), tier 2 (rows of more than
        // TIER1 edges: at most m / (TIER1 + 1)), then their two counts
        const size_t n_list2 = (size_t)m / (TIER1 + 1) + 1;
        const size_t t_list = t; t = align_up(t + ((size_t)n + n_list2 + 2) * 4);
        // the pinned control block of the arena doubles as the host side of the checks
        TRY(cudaMallocHost(&a->host_ctrl, sizeof(Ctrl)));
        TRY(cudaMallocAsync((void **)&tmp, t, s));
        long long *rp64 = (long long *)(tmp + t_rp);
        long long *rrp64 = (long long *)(tmp + t_rrp);
        unsigned *dflags = (unsigned *)(tmp + t_flags);
        unsigned long long *dhash = (unsigned long long *)(tmp + t_flags + 16);
        int *scan_scratch = (int *)(tmp + t_scan);
        int *fill = (int *)(tmp + t_fill);
        int *list1 = (int *)(tmp + t_list);
        int *list2 = list1 + n;
        int *long_cnt = list2 + n_list2;

        TRY(cudaMemsetAsync(dflags, 0, 64, s));
        TRY(cudaMemcpyAsync(rp64, row_ptr, ((size_t)n + 1) * 8, kind, s));
        TRY(cudaMemcpyAsync(dcol, col, (size_t)m * 4, kind, s));
        TRY(cudaMemcpyAsync(dw, w, (size_t)m * 4, kind, s));
        TRY(cudaMemcpyAsync(down, owner_bits, words * 4, kind, s));
        {
            const int g = (int)std::min<long long>(((long long)n + 256) / 256, 8192);
            const int ge = (int)std::min<long long>(((long long)m + 255) / 256, 8192);
            k_check_rows<<<g, 256, 0, s>>>(rp64, n, m, rp32, dflags);
            k_check_cols<<<ge, 256, 0, s>>>(dcol, m, n, dflags, BAD_COL);
            TRY(cudaGetLastError());
            if (have_rev) {
                TRY(cudaMemcpyAsync(rrp64, rrow_ptr, ((size_t)n + 1) * 8, kind, s));
                TRY(cudaMemcpyAsync(drcol, rcol, (size_t)m * 4, kind, s));
                TRY(cudaMemcpyAsync(drw, rw, (size_t)m * 4, kind, s));
                k_check_rows<<<g, 256, 0, s>>>(rrp64, n, m, rrp32, dflags + 1);
                k_check_cols<<<ge, 256, 0, s>>>((const int *)drcol, m, n, dflags, BAD_RCOL);
                TRY(cudaGetLastError());
            }
            hflags = (unsigned *)a->host_ctrl;
            TRY(cudaMemcpyAsync(hflags, dflags, 8, cudaMemcpyDeviceToHost, s));
            TRY(cudaStreamSynchronize(s));
            const unsigned fl = hflags[0], rfl = hflags[1] & BAD_ROWPTR;
            if (fl & (BAD_ROWPTR | BAD_COL)) {
                set_error("malformed forward CSR (%s)", (fl & BAD_ROWPTR) ? "row_ptr" : "col out of range");
                rc = EG_ERR_INVALID;
                goto fail;
            }
            if (fl & NOT_TOTAL) {
                set_error("arena is not total: some vertex has no successor");
                rc = EG_ERR_NOT_TOTAL;
                goto fail;
            }
            if (rfl || (fl & BAD_RCOL)) {
                set_error("malformed reverse CSR");
                rc = EG_ERR_INVALID;
                goto fail;
            }
            if (!have_rev) {
                TRY(cudaMemsetAsync(rrp32, 0, ((size_t)n + 1) * 4, s));
                k_count_in<<<ge, 256, 0, s>>>(dcol, m, rrp32);
                TRY(cudaGetLastError());
                TRY(exclusive_scan(rrp32, n + 1, scan_scratch, s));
                TRY(cudaMemcpyAsync(fill, rrp32, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
                const int gt = (int)std::min<long long>(((long long)n + 255) / 256, 1 << 14);
                const int gw = (int)std::min<long long>(((long long)n + 7) / 8, 1 << 14);
                k_scatter<<<gt, 256, 0, s>>>(n, rp32, dcol, dw, down, fill, drcol, drw);
                TRY(cudaMemsetAsync(long_cnt, 0, 8, s));
                k_collect_rows<<<gt, 256, 0, s>>>(n, rp32, list1, long_cnt, list2, long_cnt + 1);
                k_scatter_long<<<num_sms_arena(a->device) * 8, 256, 0, s>>>(rp32, dcol, dw, down, list1, long_cnt,
                                                                            list2, long_cnt + 1, fill,
                                                                            drcol, drw);
                TRY(cudaGetLastError());
            } else {
                const int gw = (int)std::min<long long>(((long long)n + 7) / 8, 1 << 16);
                k_hash_fwd<<<gw, 256, 0, s>>>(n, rp32, dcol, dw, dhash);
                k_hash_rev<<<gw, 256, 0, s>>>(n, rrp32, drcol, drw, dhash + 1);
                k_tag_rcol<<<ge, 256, 0, s>>>(m, down, drcol);
                TRY(cudaGetLastError());
                TRY(cudaMemcpyAsync(hh, dhash, 16, cudaMemcpyDeviceToHost, s));
            }
            {
                const int gt = (int)std::min<long long>(((long long)n + 255) / 256, 1 << 14);
                const int gw = (int)std::min<long long>(((long long)n + 7) / 8, 1 << 14);
                k_fill_int<<<gt, 256, 0, s>>>(dwmin, n, 0x7fffffff);
                k_fill_int<<<gt, 256, 0, s>>>(dwmax, n, (int)0x80000000);
                k_row_extremes<<<gt, 256, 0, s>>>(n, rp32, dw, dwmin, dwmax);
                if (have_rev) {  // the long-row lists are made by the reverse build otherwise
                    TRY(cudaMemsetAsync(long_cnt, 0, 8, s));
                    k_collect_rows<<<gt, 256, 0, s>>>(n, rp32, list1, long_cnt, list2, long_cnt + 1);
                }
                k_row_extremes_long<<<num_sms_arena(a->device) * 8, 256, 0, s>>>(
                    rp32, dw, list1, long_cnt, list2, long_cnt + 1, dwmin, dwmax);
                TRY(cudaGetLastError());
            }
            TRY(cudaFreeAsync(tmp, s));
            tmp = nullptr;
            TRY(cudaStreamSynchronize(s));
            if (have_rev && hh[0] != hh[1]) {
                set_error("reverse CSR does not hold the same edges as the forward CSR");
                rc = EG_ERR_INVALID;
                goto fail;
            }
        }
        a->d.n = n;
        a->d.m = m;
        a->d.row_ptr = rp32;
        a->d.col = dcol;
        a->d.w = dw;
        a->d.rrow_ptr = rrp32;
        a->d.rcol = drcol;
        a->d.rw = drw;
        a->d.owner_bits = down;
        a->d.wmin = dwmin;
        a->d.wmax = dwmax;
        TRY(cudaEventCreate(&a->ev0));
        TRY(cudaEventCreate(&a->ev1));
        TRY(cudaEventCreate(&a->evk));
        long long C = 0, wm = 0;
        rc = compute_bound(a, 1, 0, &C, &wm, s);
        if (rc != EG_OK) goto fail;
    }
#undef TRY
    *out = a;
    return EG_OK;
fail:
    if (tmp) {
        cudaFreeAsync(tmp, 0);
        cudaStreamSynchronize(0);
    }
    destroy(a);
    return rc;
}

}  // namespace eg

extern "C" {

eg_status eg_create(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                    const int64_t *rrow_ptr, const int32_t *rcol, const int32_t *rw, const uint32_t *owner_bits,
                    uint32_t flags, eg_arena **out) {
    eg::clear_error();
    try {
        return eg::create(n, m, row_ptr, col, w, rrow_ptr, rcol, rw, owner_bits, flags, out);
    } catch (...) {
        eg::set_error("unexpected exception in eg_create");
        return EG_ERR_INVALID;
    }
}

eg_status eg_destroy(eg_arena *arena) {
    eg::clear_error();
    return eg::destroy(arena);
}

eg_status eg_bound(eg_arena *arena, int64_t w_scale, int64_t w_shift, int64_t *C, int64_t *max_abs_w) {
    eg::clear_error();
    if (!arena) {
        eg::set_error("arena is NULL");
        return EG_ERR_INVALID;
    }
    long long c = 0, wm = 0;
    eg_status rc = eg::compute_bound(arena, w_scale, w_shift, &c, &wm, 0);
    if (rc != EG_OK) return rc;
    if (C) *C = c;
    if (max_abs_w) *max_abs_w = wm;
    return EG_OK;
}

eg_status eg_solve_credit(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                          void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds) {
    eg::clear_error();
    if (!arena || !credits_out) {
        eg::set_error("arena and credits_out are required");
        return EG_ERR_INVALID;
    }
    try {
        return eg::solve(arena, credit_bits, w_scale, w_shift, credits_out, st, (cudaStream_t)cuda_stream,
                         max_rounds);
    } catch (...) {
        eg::set_error("unexpected exception in eg_solve_credit");
        return EG_ERR_INVALID;
    }
}

}  // extern "C"

namespace eg {
// Every edge of vertex v (one warp per vertex) must stay in v's game.
__global__ void k_check_parts(int n, const int *row_ptr, const int *col, const long long *pp, int parts,
                              unsigned *bad) {
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
        int lo = 0, hi = parts;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pp[mid] <= v) lo = mid;
            else hi = mid;
        }
        const long long a = pp[lo], b = pp[lo + 1];
        for (int k = row_ptr[v] + lane; k < row_ptr[v + 1]; k += 32)
            if (col[k] < a || col[k] >= b) atomicOr(bad, 1u);
    }
}
}  // namespace eg

extern "C" {

eg_status eg_set_parts(eg_arena *arena, int32_t parts, const int64_t *part_ptr) {
    eg::clear_error();
    if (!arena || parts < 1 || !part_ptr) {
        eg::set_error("need an arena, parts >= 1 and part_ptr");
        return EG_ERR_INVALID;
    }
    if (part_ptr[0] != 0 || part_ptr[parts] != arena->n) {
        eg::set_error("part_ptr must start at 0 and end at n");
        return EG_ERR_INVALID;
    }
    for (int k = 0; k < parts; ++k)
        if (part_ptr[k + 1] <= part_ptr[k]) {
            eg::set_error("part %d is empty or offsets decrease", k);
            return EG_ERR_INVALID;
        }
    long long *dpp = nullptr;
    unsigned *dbad = nullptr;
    unsigned hbad = 0;
    eg_status rc = EG_OK;
    if (cudaMalloc((void **)&dpp, ((size_t)parts + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&dbad, 4) != cudaSuccess) {
        eg::set_error("device allocation failed");
        rc = EG_ERR_OOM;
    } else {
        cudaMemcpy(dpp, part_ptr, ((size_t)parts + 1) * 8, cudaMemcpyHostToDevice);
        cudaMemset(dbad, 0, 4);
        const int gw = (int)std::min<long long>(((long long)arena->n + 7) / 8, 1 << 14);
        eg::k_check_parts<<<gw, 256>>>(arena->n, arena->d.row_ptr, arena->d.col, dpp, parts, dbad);
        cudaError_t e = cudaMemcpy(&hbad, dbad, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            eg::set_error("part check failed: %s", cudaGetErrorString(e));
            rc = EG_ERR_CUDA;
        } else if (hbad) {
            eg::set_error("an edge leaves its game");
            rc = EG_ERR_INVALID;
        }
    }
    if (dpp) cudaFree(dpp);
    if (dbad) cudaFree(dbad);
    if (rc == EG_OK) arena->part_ptr.assign(part_ptr, part_ptr + parts + 1);
    return rc;
}

eg_status eg_set_option(eg_arena *arena, int32_t option, int64_t value) {
    eg::clear_error();
    if (!arena) {
        eg::set_error("arena is NULL");
        return EG_ERR_INVALID;
    }
    if (value < 0 || value > (1LL << 30)) {
        eg::set_error("option value %lld out of range", (long long)value);
        return EG_ERR_INVALID;
    }
    switch (option) {
    case EG_OPT_LOCAL_WINDOWS: arena->local_windows = (int)value; break;
    case EG_OPT_LOCAL_MAXDEG: arena->local_maxdeg = (int)value; break;
    case EG_OPT_WARM_START:
        if (value > 1) {
            eg::set_error("EG_OPT_WARM_START takes 0 or 1");
            return EG_ERR_INVALID;
        }
        arena->warm_start = (int)value;
        break;
    case EG_OPT_SEED_MAX_PAIRS: arena->seed_max_pairs = value; break;
    case EG_OPT_CAP_CERTIFY: arena->cap_certify = (int)value; break;
    case EG_OPT_CERTIFY_AFTER: arena->certify_after = value; break;
    case EG_OPT_BLOCKS_PER_SM: arena->blocks_per_sm = (int)value; break;
    case EG_OPT_KICK_ROUNDS: arena->kick_rounds = value; break;
    case EG_OPT_CHUNK_EDGES: arena->chunk_edges = (int)value; break;
    case EG_OPT_SWEEPS:
        if (value > 1024) {
            eg::set_error("EG_OPT_SWEEPS takes at most 1024");
            return EG_ERR_INVALID;
        }
        arena->sweeps = (int)value;
        break;
    case EG_OPT_DUAL_K:
        if (value < 1) {
            eg::set_error("EG_OPT_DUAL_K takes at least 1");
            return EG_ERR_INVALID;
        }
        arena->dual_k = (int)value;
        break;
    case EG_OPT_SCC_ORDER:
        if (value > 1) {
            eg::set_error("EG_OPT_SCC_ORDER takes 0 or 1");
            return EG_ERR_INVALID;
        }
        arena->scc_order = (int)value;
        break;
    case EG_OPT_WAIT_LIMIT_US:
        if (value < 1) {
            eg::set_error("EG_OPT_WAIT_LIMIT_US takes at least 1");
            return EG_ERR_INVALID;
        }
        arena->wait_limit_ns = (unsigned long long)value * 1000ull;
        break;
    case EG_OPT_GRAPH:
        if (value > 1) {
            eg::set_error("EG_OPT_GRAPH takes 0 or 1");
            return EG_ERR_INVALID;
        }
        arena->use_graph = (int)value;
        break;
    default: eg::set_error("unknown option %d", option); return EG_ERR_INVALID;
    }
    return EG_OK;
}

eg_status eg_scc_info(eg_arena *arena, int64_t *components, int64_t *levels, int64_t *passes) {
    eg::clear_error();
    if (!arena) {
        eg::set_error("arena is NULL");
        return EG_ERR_INVALID;
    }
    eg_status rc = eg::scc_levels(arena, 0);
    if (rc != EG_OK) return rc;
    if (components) *components = arena->scc_count;
    if (levels) *levels = arena->scc_nlevels;
    if (passes) *passes = arena->scc_passes;
    return EG_OK;
}

eg_status eg_scc_levels(eg_arena *arena, int32_t *level_out, int32_t *component_out) {
    eg::clear_error();
    if (!arena || (!level_out && !component_out)) {
        eg::set_error("need an arena and an output");
        return EG_ERR_INVALID;
    }
    eg_status rc = eg::scc_levels(arena, 0);
    if (rc != EG_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (level_out) e = cudaMemcpy(level_out, arena->scc_level, (size_t)arena->n * 4, cudaMemcpyDefault);
    if (e == cudaSuccess && component_out)
        e = cudaMemcpy(component_out, arena->scc_comp, (size_t)arena->n * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        eg::set_error("copy of the condensation failed: %s", cudaGetErrorString(e));
        return EG_ERR_CUDA;
    }
    return EG_OK;
}

const char *eg_last_error(void) { return eg::g_err; }

const char *eg_version(void) { return "eg-gb300 0.1"; }

}  // extern "C"
