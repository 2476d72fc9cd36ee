// Request loop over many games (eg_server_create / eg_submit / eg_poll).
//
// A scheduler thread drains the request queue in batches: it admits queued
// requests in arrival order while their memory fits the device budget,
// copies their arenas into one packed device arena (vertex and edge indices
// shifted to each game's range, so the games stay disjoint), and solves all
// of them with one batched launch (the plan of eg_solve.cu): one instance per
// request, each with its own bound C and weight map.  Requests submitted
// while a batch runs wait in the queue for the next batch, which starts as
// soon as the running one ends.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
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
    std::vector<long long> credits;  // int64 with TOP = INT64_MAX
    eg_stats st{};
    Clock::time_point submitted;
    size_t need = 0;
};

static size_t request_bytes(const eg_arena *ar) {
    return (size_t)ar->m * 16 + (size_t)ar->n * 72 + 4096;
}

// ---- packing kernels: game k's arrays into the pool at vertex base vb and
// edge base eb

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

__global__ void k_pack_owner(unsigned *dst, const unsigned *src, int n, int vb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if ((src[i >> 5] >> (i & 31)) & 1u) atomicOr(dst + ((vb + i) >> 5), 1u << ((vb + i) & 31));
}

__global__ void k_set_tail(int *row_ptr, int *rrow_ptr, int n, int m) {
    row_ptr[n] = m;
    rrow_ptr[n] = m;
}

struct Server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 1;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
    // pool: one device block for the packed arena, one for the int64 result
    eg_arena pool;
    void *pool_block = nullptr;
    size_t pool_bytes = 0;
    long long *result = nullptr;
    size_t result_cap = 0;
    long long *host_result = nullptr;
    size_t host_cap = 0;
};

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

static eg_status ensure_pool(Server *S, long long n, long long m) {
    const size_t words = ((size_t)n + 31) / 32;
    const size_t need = 2 * up256(((size_t)n + 1) * 4) + 4 * up256((size_t)m * 4) + up256(words * 4) +
                        2 * up256((size_t)n * 4);
    if (need > S->pool_bytes) {
        if (S->pool_block) cudaFree(S->pool_block);
        S->pool_block = nullptr;
        S->pool_bytes = 0;
        EG_CUDA_TRY(cudaMalloc(&S->pool_block, need));
        S->pool_bytes = need;
    }
    char *b = (char *)S->pool_block;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = b + off;
        off += up256(bytes);
        return p;
    };
    DevArena &d = S->pool.d;
    d.n = (int)n;
    d.m = (int)m;
    d.row_ptr = (int *)take(((size_t)n + 1) * 4);
    d.col = (int *)take((size_t)m * 4);
    d.w = (int *)take((size_t)m * 4);
    d.rrow_ptr = (int *)take(((size_t)n + 1) * 4);
    d.rcol = (unsigned *)take((size_t)m * 4);
    d.rw = (int *)take((size_t)m * 4);
    d.owner_bits = (unsigned *)take(words * 4);
    d.wmin = (int *)take((size_t)n * 4);
    d.wmax = (int *)take((size_t)n * 4);
    S->pool.n = (int)n;
    S->pool.m = (int)m;
    if ((size_t)n > S->result_cap) {
        if (S->result) cudaFree(S->result);
        S->result = nullptr;
        S->result_cap = 0;
        EG_CUDA_TRY(cudaMalloc((void **)&S->result, (size_t)n * 8));
        S->result_cap = (size_t)n;
    }
    if ((size_t)n > S->host_cap) {
        if (S->host_result) cudaFreeHost(S->host_result);
        S->host_result = nullptr;
        S->host_cap = 0;
        EG_CUDA_TRY(cudaMallocHost((void **)&S->host_result, (size_t)n * 8));
        S->host_cap = (size_t)n;
    }
    return EG_OK;
}

static eg_status run_batch(Server *S, std::vector<Request *> &batch) {
    long long n = 0, m = 0;
    for (Request *r : batch) {
        n += r->ar->n;
        m += r->ar->m;
    }
    if (n >= (1LL << 31) - 1 || m >= (1LL << 31) - 1) {
        set_error("batch too large for int32 indices");
        return EG_ERR_INVALID;
    }
    eg_status rc = ensure_pool(S, n, m);
    if (rc != EG_OK) return rc;
    cudaStream_t s = S->stream;
    DevArena &d = S->pool.d;
    EG_CUDA_TRY(cudaMemsetAsync((void *)d.owner_bits, 0, (((size_t)n + 31) / 32) * 4, s));
    S->pool.part_ptr.assign(1, 0);
    long long vb = 0, eb = 0;
    for (Request *r : batch) {
        const DevArena &a = r->ar->d;
        const int g1 = (int)std::min<long long>((a.n + 255) / 256, 4096);
        const int g2 = (int)std::min<long long>((a.m + 255) / 256, 8192);
        k_pack_rows<<<g1, 256, 0, s>>>((int *)d.row_ptr + vb, a.row_ptr, a.n, (int)eb);
        k_pack_rows<<<g1, 256, 0, s>>>((int *)d.rrow_ptr + vb, a.rrow_ptr, a.n, (int)eb);
        k_pack_cols<<<g2, 256, 0, s>>>((int *)d.col + eb, a.col, a.m, (int)vb);
        k_pack_rcols<<<g2, 256, 0, s>>>((unsigned *)d.rcol + eb, a.rcol, a.m, (int)vb);
        k_pack_owner<<<g1, 256, 0, s>>>((unsigned *)d.owner_bits, a.owner_bits, a.n, (int)vb);
        EG_CUDA_TRY(cudaGetLastError());
        EG_CUDA_TRY(cudaMemcpyAsync((int *)d.w + eb, a.w, (size_t)a.m * 4, cudaMemcpyDeviceToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync((int *)d.rw + eb, a.rw, (size_t)a.m * 4, cudaMemcpyDeviceToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync((int *)d.wmin + vb, a.wmin, (size_t)a.n * 4, cudaMemcpyDeviceToDevice, s));
        EG_CUDA_TRY(cudaMemcpyAsync((int *)d.wmax + vb, a.wmax, (size_t)a.n * 4, cudaMemcpyDeviceToDevice, s));
        vb += a.n;
        eb += a.m;
        S->pool.part_ptr.push_back(vb);
    }
    k_set_tail<<<1, 1, 0, s>>>((int *)d.row_ptr, (int *)d.rrow_ptr, (int)n, (int)m);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaStreamSynchronize(s));

    const int k = (int)batch.size();
    std::vector<int32_t> part(k);
    std::vector<int64_t> sc(k), sh(k);
    bool want64 = false;
    for (int i = 0; i < k; ++i) {
        part[i] = i;
        sc[i] = batch[i]->scale;
        sh[i] = batch[i]->shift;
        want64 = want64 || batch[i]->credit_bits == 64;
    }
    eg_plan_impl *plan = nullptr;
    rc = plan_create(&S->pool, k, part.data(), sc.data(), sh.data(), want64 ? 64 : 0, &plan);
    if (rc != EG_OK) return rc;
    eg_stats st{};
    rc = plan_run(plan, S->result, &st, s, 0);
    if (rc == EG_OK) {
        cudaError_t e = cudaMemcpyAsync(S->host_result, S->result, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("result copy failed: %s", cudaGetErrorString(e));
            rc = EG_ERR_CUDA;
        }
    }
    if (rc == EG_OK) {
        for (int i = 0; i < k; ++i) {
            long long off = 0, len = 0, C = 0;
            int bits_alone = 32;
            plan_instance_info(plan, i, &off, &len, &C, &bits_alone);
            Request *r = batch[i];
            r->st = st;
            r->st.C = C;
            r->st.fixpoint_ms = st.ms;
            if (r->credit_bits == 32 && bits_alone == 64) {
                r->status = EG_ERR_OVERFLOW;
                continue;
            }
            r->st.credit_bits = r->credit_bits == 32 ? 32 : 64;
            r->credits.assign(S->host_result + off, S->host_result + off + len);
        }
    }
    plan_release(plan);
    return rc;
}

static void worker_main(Server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop) return;
            size_t mem = 0;
            while (!S->queue.empty() && (int)batch.size() < S->max_batch) {
                Request *r = S->queue.front();
                if (r->need > S->budget) {
                    S->queue.pop_front();
                    r->status = EG_ERR_OOM;
                    r->st.status = EG_ERR_OOM;
                    r->done = true;
                    continue;
                }
                if (mem + r->need > S->budget && !batch.empty()) break;
                S->queue.pop_front();
                batch.push_back(r);
                mem += r->need;
            }
            if (batch.empty()) {
                S->done_cv.notify_all();
                continue;
            }
        }
        const eg_status rc = run_batch(S, batch);
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request *r : batch) {
                if (rc != EG_OK && r->status == EG_OK) r->status = rc;
                r->st.status = r->status;
                r->st.ms = std::chrono::duration<double, std::milli>(now - r->submitted).count();
                r->done = true;
            }
        }
        S->done_cv.notify_all();
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
    S->max_batch = max_batch;
    cudaGetDevice(&S->device);
    S->pool.device = S->device;
    S->pool.use_graph = 0;  // a new packing every batch: nothing to replay
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->pool.ev0) != cudaSuccess || cudaEventCreate(&S->pool.ev1) != cudaSuccess ||
        cudaEventCreate(&S->pool.evk) != cudaSuccess || cudaMallocHost(&S->pool.host_ctrl, sizeof(eg::Ctrl)) != cudaSuccess) {
        eg::set_error("server set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        eg_server_destroy(S);
        return EG_ERR_CUDA;
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
    r->need = eg::request_bytes(arena);
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
        *ticket = r->ticket;
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
        const size_t n = r->credits.size();
        std::vector<int32_t> narrow;
        const void *src = r->credits.data();
        size_t bytes = n * 8;
        if (r->credit_bits == 32) {
            narrow.resize(n);
            for (size_t i = 0; i < n; ++i)
                narrow[i] = r->credits[i] == INT64_MAX ? INT32_MAX : (int32_t)r->credits[i];
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
    delete r;
    return rc;
}

eg_status eg_server_destroy(eg_server *S) {
    eg::clear_error();
    if (!S) return EG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->all) delete kv.second;
    S->all.clear();
    S->queue.clear();
    if (S->pool_block) cudaFree(S->pool_block);
    if (S->result) cudaFree(S->result);
    if (S->host_result) cudaFreeHost(S->host_result);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->pool.ev0) cudaEventDestroy(S->pool.ev0);
    if (S->pool.ev1) cudaEventDestroy(S->pool.ev1);
    if (S->pool.evk) cudaEventDestroy(S->pool.evk);
    if (S->pool.host_ctrl) cudaFreeHost(S->pool.host_ctrl);
    S->pool.host_ctrl = nullptr;
    S->pool.ev0 = S->pool.ev1 = S->pool.evk = nullptr;
    delete S;
    return EG_OK;
}

}  // extern "C"
