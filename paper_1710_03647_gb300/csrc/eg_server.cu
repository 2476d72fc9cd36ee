// Request loop over many games (eg_server_create / eg_submit / eg_poll)
// with continuous batching.
//
// The server owns a pool arena sized from its device memory budget and one
// resident solve state over it (eg_solve.cu).  A scheduler thread admits
// queued requests in arrival order whenever a slot and room in the pool are
// free: it copies the request's arena into a free vertex range and edge
// range of the pool (indices shifted to the range, so the games stay
// disjoint), computes its bound C, and appends its initial push list to the
// round the resident solve is at.  It then runs the persistent fixpoint for
// a slice of rounds over every resident game at once.  A slice ends after a
// fixed number of rounds, when no work is left, or as soon as eg_submit rings
// the doorbell, so a new request joins the running solve at the next round
// instead of waiting for the others to finish.  After each slice, a game with
// no entry left in the round's lists is finished: its credits are copied
// by DMA into a pinned result buffer (reused across requests), its ranges and
// slot are freed, and waiting requests take them.
//
// A game of at least SOLO_EDGES edges fills the GPU by itself, so sharing the
// resident solve gains it nothing: it skips the pool and is solved alone
// (eg_solve_credit's route) between slices, straight into its result buffer.
//
// A game still unfinished after its arena's EG_OPT_CERTIFY_AFTER rounds (with
// certified trial caps on) is taken out: it is solved alone with the trials
// (eg_solve_credit's route), and its slot is retired -- its views get a
// negative C, so the fixpoint kernel consumes its remaining entries without
// work -- and freed once no entry of it is left.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    eg_arena *ar = nullptr;
    int credit_bits = 0;
    long long scale = 1, shift = 0;
    bool done = false;
    eg_status status = EG_OK;
    // the credits, in a pinned buffer from the server's pool: n elements of
    // res_w bytes (int32 with TOP = INT32_MAX, or int64 with TOP = INT64_MAX)
    void *res = nullptr;
    int res_cls = -1, res_w = 8;
    size_t res_n = 0;
    eg_stats st{};
    Clock::time_point submitted;
    // placement while resident
    int slot = -1;
    long long vb = 0, eb = 0;
    long long C = 0;
    long long r_admit = 0;
    bool tried_alone = false;  // took the idle route's short attempt already
    unsigned long long relax0 = 0, lifts0 = 0, pushes0 = 0, enq0 = 0;
    double dev_ms = 0;
};

// Pinned host buffers for finished credits, kept by power-of-two size class
// and reused: results land in them by DMA and stay until eg_poll copies them
// out, so the worker never copies credits on the host.
struct PinPool {
    std::mutex mu;
    std::vector<std::vector<void *>> free_;  // by class: 2^c bytes
    std::vector<void *> all;
    void *get(size_t bytes, int *cls) {
        int c = 15;
        while (((size_t)1 << c) < bytes) ++c;
        *cls = c;
        {
            std::lock_guard<std::mutex> lk(mu);
            if ((int)free_.size() > c && !free_[c].empty()) {
                void *p = free_[c].back();
                free_[c].pop_back();
                return p;
            }
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, (size_t)1 << c) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lk(mu);
        all.push_back(p);
        return p;
    }
    void put(void *p, int cls) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu);
        if ((int)free_.size() <= cls) free_.resize(cls + 1);
        free_[cls].push_back(p);
    }
    void release_all() {
        for (void *p : all) cudaFreeHost(p);
        all.clear();
        free_.clear();
    }
};

// Takes a result buffer of n elements of w bytes for r from the pool.
static eg_status take_result(PinPool &pins, Request *r, size_t n, int w) {
    r->res = pins.get(std::max<size_t>(n, 1) * w, &r->res_cls);
    if (!r->res) {
        set_error("pinned result buffer of %zu bytes failed", n * w);
        return EG_ERR_OOM;
    }
    r->res_n = n;
    r->res_w = w;
    return EG_OK;
}

static void drop_result(PinPool &pins, Request *r) {
    pins.put(r->res, r->res_cls);
    r->res = nullptr;
    r->res_cls = -1;
    r->res_n = 0;
}

// First-fit allocator of index ranges, merging freed neighbours.
struct RangeAlloc {
    std::map<long long, long long> free_;  // start -> length
    void init(long long cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    long long alloc(long long len) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < len) continue;
            const long long st = it->first, l = it->second;
            free_.erase(it);
            if (l > len) free_[st + len] = l - len;
            return st;
        }
        return -1;
    }
    void release(long long st, long long len) {
        if (len <= 0) return;
        auto it = free_.emplace(st, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// device bytes per pool vertex (arena rows, weight extremes, owner bit and
// the int64 solve state with its lists, bitmaps and slot ids) and per edge
constexpr size_t POOL_VERTEX_BYTES = 74;
constexpr size_t POOL_EDGE_BYTES = 16;
constexpr long long SLICE_ROUNDS = 32;
// A game with at least this many edges fills the GPU on its own: it is solved
// alone (eg_solve_credit's route) between slices instead of joining the pool.
constexpr long long SOLO_EDGES = 1LL << 19;

__global__ void k_pack_rows(int *dst, const int *src, int n, int add) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] + add;
}

__global__ void k_pack_cols(int *dst, const int *src, int m, int add) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) dst[i] = src[i] + add;
}

__global__ void k_pack_rcols(unsigned *dst, const unsigned *src, int m, int add) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const unsigned r = src[i];
        dst[i] = ((r & 0x7fffffffu) + (unsigned)add) | (r & P1_FLAG);
    }
}

// owner bits of game vertices [0, n) to pool bits [vb, vb + n); the range's
// old bits were cleared first (k_unset_bits)
__global__ void k_pack_owner(unsigned *dst, const unsigned *src, int n, int vb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if ((src[i >> 5] >> (i & 31)) & 1u) atomicOr(dst + ((vb + i) >> 5), 1u << ((vb + i) & 31));
}

__global__ void k_unset_bits(unsigned *bits, int g0, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAnd(bits + ((g0 + i) >> 5), ~(1u << ((g0 + i) & 31)));
}

// A slot whose game was solved elsewhere, freed once its entries are gone.
struct Retiring {
    int slot;
    long long vb, nv, eb, m;
};

struct Server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the pool: vertex slots [0, NV) and edges [0, NE); a game of n vertices
    // takes n + 1 vertex slots (its last row offset sits in the extra one)
    long long NV = 0, NE = 0;
    void *pool_block = nullptr;
    DevArena pool{};
    RangeAlloc vfree, efree;
    std::vector<int> free_slots;
    std::vector<Request *> active;  // by slot
    int nactive = 0;
    std::vector<Retiring> retiring;
    Resident R;
    PinPool pins;  // result buffers
    long long fail_reservations = 0;  // test hook: reservations still to refuse
    int idle_solo = 1;                // a lone request on an idle server gets a short attempt alone
    eg_server_counters ctr{};         // under mu
};

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

static eg_status create_pool(Server *S) {
    const long long NV = S->NV, NE = S->NE;
    const size_t words = ((size_t)NV + 31) / 32;
    const size_t bytes = 2 * up256(((size_t)NV + 1) * 4) + 4 * up256((size_t)NE * 4) + up256(words * 4) +
                         2 * up256((size_t)NV * 4);
    EG_CUDA_TRY(cudaMalloc(&S->pool_block, bytes));
    EG_CUDA_TRY(cudaMemsetAsync(S->pool_block, 0, bytes, S->stream));
    char *b = (char *)S->pool_block;
    size_t off = 0;
    auto take = [&](size_t n) {
        char *p = b + off;
        off += up256(n);
        return p;
    };
    DevArena &d = S->pool;
    d.n = (int)NV;
    d.m = (int)NE;
    d.row_ptr = (int *)take(((size_t)NV + 1) * 4);
    d.col = (int *)take((size_t)NE * 4);
    d.w = (int *)take((size_t)NE * 4);
    d.rrow_ptr = (int *)take(((size_t)NV + 1) * 4);
    d.rcol = (unsigned *)take((size_t)NE * 4);
    d.rw = (int *)take((size_t)NE * 4);
    d.owner_bits = (unsigned *)take(words * 4);
    d.wmin = (int *)take((size_t)NV * 4);
    d.wmax = (int *)take((size_t)NV * 4);
    eg_status rc = resident_create(S->R, S->device, (int)NV, S->max_slots, S->stream);
    if (rc != EG_OK) return rc;
    S->R.A = S->pool;
    S->vfree.init(NV);
    S->efree.init(NE);
    S->free_slots.clear();
    for (int k = S->max_slots - 1; k >= 0; --k) S->free_slots.push_back(k);
    S->active.assign(S->max_slots, nullptr);
    return EG_OK;
}

// Copies the request's arena into its pool ranges and joins it to the solve.
static eg_status place(Server *S, Request *r) {
    cudaStream_t s = S->stream;
    const DevArena &a = r->ar->d;
    DevArena &d = S->pool;
    const int vb = (int)r->vb, eb = (int)r->eb;
    const int g1 = (int)std::min<long long>((a.n + 256) / 256, 4096);
    const int g2 = (int)std::min<long long>((a.m + 255) / 256, 8192);
    k_pack_rows<<<g1, 256, 0, s>>>((int *)d.row_ptr + vb, a.row_ptr, a.n + 1, eb);
    k_pack_rows<<<g1, 256, 0, s>>>((int *)d.rrow_ptr + vb, a.rrow_ptr, a.n + 1, eb);
    k_pack_cols<<<g2, 256, 0, s>>>((int *)d.col + eb, a.col, a.m, vb);
    k_pack_rcols<<<g2, 256, 0, s>>>((unsigned *)d.rcol + eb, a.rcol, a.m, vb);
    k_unset_bits<<<g1, 256, 0, s>>>((unsigned *)d.owner_bits, vb, a.n + 1);
    k_pack_owner<<<g1, 256, 0, s>>>((unsigned *)d.owner_bits, a.owner_bits, a.n, vb);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemcpyAsync((int *)d.w + eb, a.w, (size_t)a.m * 4, cudaMemcpyDeviceToDevice, s));
    EG_CUDA_TRY(cudaMemcpyAsync((int *)d.rw + eb, a.rw, (size_t)a.m * 4, cudaMemcpyDeviceToDevice, s));
    EG_CUDA_TRY(cudaMemcpyAsync((int *)d.wmin + vb, a.wmin, (size_t)a.n * 4, cudaMemcpyDeviceToDevice, s));
    EG_CUDA_TRY(cudaMemcpyAsync((int *)d.wmax + vb, a.wmax, (size_t)a.n * 4, cudaMemcpyDeviceToDevice, s));
    long long C = 0, wmax = 0;
    eg_status rc = compute_bound(r->ar, r->scale, r->shift, &C, &wmax, s);
    if (rc != EG_OK) return rc;
    if (r->credit_bits == 32 && C + wmax > 0x7fffffffLL - 1) {
        set_error("int32 credits cannot hold C + max|w'| = %lld", C + wmax);
        return EG_ERR_OVERFLOW;
    }
    r->C = C;
    rc = resident_admit(S->R, r->slot, vb, a.n, r->scale, r->shift, C, s);
    if (rc != EG_OK) return rc;
    const Ctrl *hc = (const Ctrl *)S->R.host_ctrl;
    r->r_admit = S->R.r;
    r->relax0 = hc->relax;
    r->lifts0 = hc->lifts;
    r->pushes0 = hc->pushes;
    r->enq0 = hc->enqueues;
    return EG_OK;
}

static void release(Server *S, Request *r) {
    S->vfree.release(r->vb, (long long)r->ar->n + 1);
    S->efree.release(r->eb, r->ar->m);
    if (r->slot >= 0) {
        S->active[r->slot] = nullptr;
        S->free_slots.push_back(r->slot);
        r->slot = -1;
    }
}

// Marks requests done (under the lock) and wakes pollers.
static void complete(Server *S, std::vector<Request *> &fin) {
    if (fin.empty()) return;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request *r : fin) {
            r->st.status = r->status;
            r->st.ms = std::chrono::duration<double, std::milli>(now - r->submitted).count();
            r->done = true;
            ++S->ctr.completed;
        }
    }
    S->done_cv.notify_all();
    fin.clear();
}

// Solves a large game alone (eg_solve_credit's route, int32 when it fits)
// straight into its pinned result buffer and completes its request.
static void solo(Server *S, Request *r, std::vector<Request *> &fin) {
    const size_t n = (size_t)r->ar->n;
    const int w = r->credit_bits == 32 ? 4 : 8;
    eg_stats st{};
    eg_status rc = take_result(S->pins, r, n, w);
    if (rc == EG_OK) rc = solve(r->ar, r->credit_bits, r->scale, r->shift, r->res, &st, S->stream, 0);
    r->status = rc;
    if (rc == EG_OK)
        r->st = st;
    else
        drop_result(S->pins, r);
    fin.push_back(r);
}

// The idle route: a request that found the server idle gets the single-game
// route's first attempt alone (EG_OPT_CERTIFY_AFTER rounds, 8 if that is 0).
// Returns true if that settled it (solved or failed), false if it needs more
// rounds; then it goes to the pool like any other request.
static bool idle_attempt(Server *S, Request *r, std::vector<Request *> &fin) {
    r->tried_alone = true;
    const long long rounds = r->ar->certify_after > 0 ? r->ar->certify_after : 8;
    eg_stats st{};
    eg_status rc = take_result(S->pins, r, (size_t)r->ar->n, r->credit_bits == 32 ? 4 : 8);
    if (rc == EG_OK) rc = solve(r->ar, r->credit_bits, r->scale, r->shift, r->res, &st, S->stream, 0, rounds);
    if (rc == EG_ERR_BUDGET) {
        drop_result(S->pins, r);
        return false;
    }
    r->status = rc;
    if (rc == EG_OK) {
        r->st = st;
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->ctr.solo;
        ++S->ctr.idle_solo;
    } else {
        drop_result(S->pins, r);
    }
    fin.push_back(r);
    return true;
}

// Solves a slow resident game alone with certified trial caps, then retires
// its slot (views with C < 0: the kernel drops its entries).
static eg_status take_out(Server *S, Request *r, std::vector<Request *> &fin) {
    eg_stats st{};
    eg_status rc = take_result(S->pins, r, (size_t)r->ar->n, 8);
    if (rc == EG_OK) rc = solve(r->ar, 64, r->scale, r->shift, r->res, &st, S->stream, 0);
    r->status = rc;
    if (rc != EG_OK) drop_result(S->pins, r);
    if (rc == EG_OK) {
        st.credit_bits = r->credit_bits == 32 ? 32 : 64;
        st.rounds += S->R.r - r->r_admit;
        st.fixpoint_ms += r->dev_ms;
        r->st = st;
    }
    const long long retired = -1;
    EG_CUDA_TRY(cudaMemcpyAsync(S->R.C + r->slot, &retired, 8, cudaMemcpyHostToDevice, S->stream));
    EG_CUDA_TRY(cudaStreamSynchronize(S->stream));
    S->retiring.push_back(Retiring{r->slot, r->vb, (long long)r->ar->n + 1, r->eb, r->ar->m});
    S->active[r->slot] = nullptr;
    r->slot = -1;
    --S->nactive;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->ctr.taken_out;
    }
    fin.push_back(r);
    return EG_OK;
}

static eg_status harvest(Server *S, std::vector<Request *> &fin) {
    eg_status rc = resident_busy(S->R, S->stream);
    if (rc != EG_OK) return rc;
    // retired slots with no entry left are free again
    for (size_t k = 0; k < S->retiring.size();) {
        const Retiring t = S->retiring[k];
        if (S->R.host_busy[t.slot]) {
            ++k;
            continue;
        }
        S->vfree.release(t.vb, t.nv);
        S->efree.release(t.eb, t.m);
        S->free_slots.push_back(t.slot);
        S->retiring[k] = S->retiring.back();
        S->retiring.pop_back();
    }
    std::vector<Request *> ready;
    for (int k = 0; k < S->max_slots; ++k) {
        Request *r = S->active[k];
        if (r && !S->R.host_busy[k]) ready.push_back(r);
    }
    // games that are slow in the resident solve go through the certified route
    for (int k = 0; k < S->max_slots; ++k) {
        Request *r = S->active[k];
        if (!r || !S->R.host_busy[k]) continue;
        const eg_arena *ar = r->ar;
        if (ar->cap_certify > 0 && ar->warm_start && ar->certify_after > 0 &&
            S->R.r - r->r_admit >= ar->certify_after) {
            rc = take_out(S, r, fin);
            if (rc != EG_OK) return rc;
        }
    }
    // a game whose pinned result buffer cannot be had now stays resident (it
    // has no work left) and is collected at a later harvest
    for (size_t k = 0; k < ready.size();) {
        if (take_result(S->pins, ready[k], (size_t)ready[k]->ar->n, 8) != EG_OK) {
            ready[k] = ready.back();
            ready.pop_back();
            continue;
        }
        ++k;
    }
    if (ready.empty()) return EG_OK;
    for (Request *r : ready)
        EG_CUDA_TRY(cudaMemcpyAsync(r->res, (const long long *)S->R.sb.d.f + r->vb, (size_t)r->ar->n * 8,
                                    cudaMemcpyDeviceToHost, S->stream));
    EG_CUDA_TRY(cudaStreamSynchronize(S->stream));
    const Ctrl *hc = (const Ctrl *)S->R.host_ctrl;
    for (Request *r : ready) {
        r->st = eg_stats{};
        r->st.C = r->C;
        r->st.credit_bits = r->credit_bits == 32 ? 32 : 64;
        r->st.rounds = S->R.r - r->r_admit;
        r->st.lifts = (int64_t)(hc->lifts - r->lifts0);
        r->st.pushes = (int64_t)(hc->pushes - r->pushes0);
        r->st.relaxations = (int64_t)(hc->relax - r->relax0);
        r->st.enqueues = (int64_t)(hc->enqueues - r->enq0);
        r->st.fixpoint_ms = r->dev_ms;
        r->status = EG_OK;
        release(S, r);
        --S->nactive;
        fin.push_back(r);
    }
    return EG_OK;
}

static void fail_active(Server *S, eg_status rc, std::vector<Request *> &fin) {
    for (const Retiring &t : S->retiring) {  // the state is reset after a failure
        S->vfree.release(t.vb, t.nv);
        S->efree.release(t.eb, t.m);
        S->free_slots.push_back(t.slot);
    }
    S->retiring.clear();
    for (int k = 0; k < S->max_slots; ++k) {
        Request *r = S->active[k];
        if (!r) continue;
        r->status = rc;
        release(S, r);
        --S->nactive;
        fin.push_back(r);
    }
}

static void worker_main(Server *S) {
    cudaSetDevice(S->device);
    std::vector<Request *> fin;
    for (;;) {
        std::vector<Request *> admitted, alone, idle;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->queue.empty() || S->nactive > 0 || !S->retiring.empty(); });
            if (S->stop) break;
            while (!S->queue.empty()) {
                Request *r = S->queue.front();
                const long long nv = (long long)r->ar->n + 1, m = r->ar->m;
                if (nv > S->NV || m > S->NE) {  // can never fit the budget
                    S->queue.pop_front();
                    r->status = EG_ERR_OOM;
                    fin.push_back(r);
                    continue;
                }
                if (m >= SOLO_EDGES) {  // fills the GPU alone: no slot, solved between slices
                    S->queue.pop_front();
                    ++S->ctr.solo;
                    alone.push_back(r);
                    continue;
                }
                // the only request, and nothing resident: the device is idle, so
                // a short attempt alone answers most games without the pool copy
                // and the slice round trip
                if (S->idle_solo && !r->tried_alone && S->nactive == 0 && S->retiring.empty() && admitted.empty() &&
                    alone.empty() && idle.empty() && S->queue.size() == 1) {
                    S->queue.pop_front();
                    idle.push_back(r);
                    continue;
                }
                if (S->free_slots.empty()) break;
                if (S->fail_reservations > 0) {  // injected: the pool reports no room
                    --S->fail_reservations;
                    ++S->ctr.refused;
                    break;
                }
                const long long vb = S->vfree.alloc(nv);
                if (vb < 0) {
                    ++S->ctr.refused;
                    break;
                }
                const long long eb = S->efree.alloc(m);
                if (eb < 0) {
                    S->vfree.release(vb, nv);
                    ++S->ctr.refused;
                    break;
                }
                S->queue.pop_front();
                r->vb = vb;
                r->eb = eb;
                r->slot = S->free_slots.back();
                S->free_slots.pop_back();
                S->active[r->slot] = r;
                ++S->nactive;
                ++S->ctr.admitted;
                admitted.push_back(r);
            }
            *(volatile unsigned *)S->R.bell_host = 0;  // a later eg_submit rings again
        }
        for (Request *r : admitted) {
            const eg_status rc = place(S, r);
            if (rc != EG_OK) {
                r->status = rc;
                release(S, r);
                --S->nactive;
                fin.push_back(r);
            }
        }
        for (Request *r : alone) {
            solo(S, r, fin);
            complete(S, fin);
        }
        for (Request *r : idle) {
            if (idle_attempt(S, r, fin)) {
                complete(S, fin);
                continue;
            }
            // unfinished: back to the front of the queue, to join the pool
            std::lock_guard<std::mutex> lk(S->mu);
            S->queue.push_front(r);
        }
        complete(S, fin);
        if (S->nactive == 0 && S->retiring.empty()) continue;
        int dev = DEV_OK;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            ++S->ctr.slices;
        }
        cudaEventRecord(S->e0, S->stream);
        eg_status rc = resident_slice(S->R, SLICE_ROUNDS, S->stream, &dev);
        cudaEventRecord(S->e1, S->stream);
        if (rc == EG_OK && dev != DEV_OK) {
            set_error("a device-side wait exceeded its limit");
            rc = EG_ERR_TIMEOUT;
        }
        if (rc == EG_OK) {
            cudaEventSynchronize(S->e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, S->e0, S->e1);
            for (Request *r : S->active)
                if (r) r->dev_ms += ms;
            rc = harvest(S, fin);
        }
        if (rc != EG_OK) {
            fail_active(S, rc, fin);
            resident_reset(S->R, S->stream);
        }
        complete(S, fin);
    }
}

}  // namespace eg

struct eg_server : eg::Server {};

extern "C" {

eg_status eg_server_create(size_t device_mem_budget, int32_t max_batch, eg_server **out) {
    eg::clear_error();
    if (!out || max_batch < 1 || device_mem_budget == 0) {
        eg::set_error("need out, max_batch >= 1 and a non-zero budget");
        return EG_ERR_INVALID;
    }
    *out = nullptr;
    eg_server *S = new (std::nothrow) eg_server();
    if (!S) {
        eg::set_error("host allocation failed");
        return EG_ERR_OOM;
    }
    S->budget = device_mem_budget;
    S->max_slots = max_batch;
    cudaGetDevice(&S->device);
    // split the budget between vertex slots and edges in the proportion of
    // a game with about 8 edges per vertex
    const double vb = 0.35 * (double)device_mem_budget / eg::POOL_VERTEX_BYTES;
    const double ebytes = 0.65 * (double)device_mem_budget / eg::POOL_EDGE_BYTES;
    S->NV = (long long)std::min(vb, (double)((1LL << 31) - 64));
    S->NE = (long long)std::min(ebytes, (double)((1LL << 31) - 64));
    if (S->NV < 2 || S->NE < 1) {
        eg::set_error("budget too small for any game");
        delete S;
        return EG_ERR_INVALID;
    }
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->e0) != cudaSuccess || cudaEventCreate(&S->e1) != cudaSuccess) {
        eg::set_error("server set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        eg_server_destroy(S);
        return EG_ERR_CUDA;
    }
    eg_status prc = eg::create_pool(S);
    if (prc != EG_OK) {
        eg_server_destroy(S);
        return prc;
    }
    try {
        S->worker = std::thread(eg::worker_main, (eg::Server *)S);
    } catch (...) {
        eg::set_error("could not start the scheduler thread");
        eg_server_destroy(S);
        return EG_ERR_INVALID;
    }
    *out = S;
    return EG_OK;
}

eg_status eg_submit(eg_server *S, eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                    uint64_t *ticket) {
    eg::clear_error();
    if (!S || !arena || !ticket) {
        eg::set_error("server, arena and ticket are required");
        return EG_ERR_INVALID;
    }
    if (credit_bits != 0 && credit_bits != 32 && credit_bits != 64) {
        eg::set_error("credit_bits must be 0, 32 or 64");
        return EG_ERR_INVALID;
    }
    const long long sa = w_scale < 0 ? -w_scale : w_scale, sh = w_shift < 0 ? -w_shift : w_shift;
    if (sa > (1LL << 30) || sh > (1LL << 61)) {
        eg::set_error("weight map out of range");
        return EG_ERR_INVALID;
    }
    eg::Request *r = new (std::nothrow) eg::Request();
    if (!r) {
        eg::set_error("host allocation failed");
        return EG_ERR_OOM;
    }
    r->ar = arena;
    r->credit_bits = credit_bits;
    r->scale = w_scale;
    r->shift = w_shift;
    r->submitted = eg::Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            eg::set_error("server is shutting down");
            return EG_ERR_BUSY;
        }
        r->ticket = S->next_ticket++;
        S->all[r->ticket] = r;
        S->queue.push_back(r);
        ++S->ctr.submitted;
        *ticket = r->ticket;
        if (S->R.bell_host) *(volatile unsigned *)S->R.bell_host = 1;  // end the running slice early
    }
    S->cv.notify_one();
    return EG_OK;
}

eg_status eg_poll(eg_server *S, uint64_t ticket, void *credits_out, eg_stats *st) {
    eg::clear_error();
    if (!S) {
        eg::set_error("server is NULL");
        return EG_ERR_INVALID;
    }
    eg::Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end()) {
            eg::set_error("unknown ticket %llu", (unsigned long long)ticket);
            return EG_ERR_INVALID;
        }
        if (!it->second->done) return EG_PENDING;
        r = it->second;
        S->all.erase(it);
    }
    eg_status rc = r->status;
    if (rc == EG_OK && credits_out) {
        const size_t n = r->res_n;
        std::vector<int32_t> narrow;
        const void *src = r->res;
        size_t bytes = n * r->res_w;
        if (r->credit_bits == 32 && r->res_w == 8) {  // int64 state, int32 answer
            const long long *wide = (const long long *)r->res;
            narrow.resize(n);
            for (size_t i = 0; i < n; ++i) narrow[i] = wide[i] == INT64_MAX ? INT32_MAX : (int32_t)wide[i];
            src = narrow.data();
            bytes = n * 4;
        }
        cudaPointerAttributes attr{};
        const bool dev = cudaPointerGetAttributes(&attr, credits_out) == cudaSuccess &&
                         (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (dev) {
            cudaError_t e = cudaMemcpy(credits_out, src, bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                eg::set_error("credit copy failed: %s", cudaGetErrorString(e));
                rc = EG_ERR_CUDA;
            }
        } else {
            memcpy(credits_out, src, bytes);
        }
    } else if (rc != EG_OK) {
        eg::set_error("request %llu failed with status %d", (unsigned long long)ticket, rc);
    }
    if (st) *st = r->st;
    drop_result(S->pins, r);
    delete r;
    return rc;
}

eg_status eg_server_set_option(eg_server *S, int32_t option, int64_t value) {
    eg::clear_error();
    if (!S || value < 0) {
        eg::set_error("need a server and a non-negative value");
        return EG_ERR_INVALID;
    }
    switch (option) {
    case EG_SRV_FAIL_RESERVATIONS: {
        std::lock_guard<std::mutex> lk(S->mu);
        S->fail_reservations = value;
        break;
    }
    case EG_SRV_IDLE_SOLO: {
        if (value > 1) {
            eg::set_error("EG_SRV_IDLE_SOLO takes 0 or 1");
            return EG_ERR_INVALID;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->idle_solo = (int)value;
        break;
    }
    default: eg::set_error("unknown server option %d", option); return EG_ERR_INVALID;
    }
    S->cv.notify_one();
    return EG_OK;
}

eg_status eg_server_counters_get(eg_server *S, eg_server_counters *out) {
    eg::clear_error();
    if (!S || !out) {
        eg::set_error("server and out are required");
        return EG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->ctr;
    return EG_OK;
}

eg_status eg_server_destroy(eg_server *S) {
    eg::clear_error();
    if (!S) return EG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        if (S->R.bell_host) *(volatile unsigned *)S->R.bell_host = 1;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (auto &kv : S->all) delete kv.second;
    S->all.clear();
    S->queue.clear();
    eg::resident_free(S->R);
    if (S->pool_block) cudaFree(S->pool_block);
    S->pins.release_all();
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->e0) cudaEventDestroy(S->e0);
    if (S->e1) cudaEventDestroy(S->e1);
    delete S;
    return EG_OK;
}

}  // extern "C"
