// Autotuner of the solver's launch settings (eg_autotune, eg_plan_autotune),
// with a cache of chosen settings on disk.
//
// The settings that change how fast the least fixpoint is reached -- never
// the result -- are the per-warp local worklist budget and its degree
// threshold, the resident blocks per SM of the persistent kernel, the first
// trial cap of the certified route and the round budget of the first
// attempt.  The best values depend on the arena: R-MAT's power-law rows
// finish in a few rounds, a road-like grid climbs for thousands of rounds
// through the certified trials.  The tuner times real solves (each one exact)
// in a coordinate search from the arena's current settings and keeps a
// candidate only if it beats the best so far by more than the noise margin.
//
// The choice is cached under a signature of the instance: log2 n, the mean
// degree, the log2 histograms of out- and in-degrees (coarse classes per
// bin), the credit width and log2(C / max|w'|), which sets how far the
// plain lifting would climb and so how much the certified trials matter.
// An instance with a cached signature takes the settings without timing.
// The cache is a text file of JSON lines, one object per signature,
// rewritten atomically (temporary file, then rename).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

constexpr int HIST_BINS = 24;

// Vertices per floor(log2(degree)) bin, out-degrees in hist[0..23] and
// in-degrees in hist[24..47] (degree 0 counts in bin 0).
__global__ void k_degree_hist(DevArena A, unsigned long long *hist) {
    __shared__ unsigned h[2 * HIST_BINS];
    for (int i = threadIdx.x; i < 2 * HIST_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        const int od = __ldg(A.row_ptr + v + 1) - __ldg(A.row_ptr + v);
        const int id = __ldg(A.rrow_ptr + v + 1) - __ldg(A.rrow_ptr + v);
        atomicAdd(&h[min(HIST_BINS - 1, od > 0 ? 31 - __clz(od) : 0)], 1u);
        atomicAdd(&h[HIST_BINS + min(HIST_BINS - 1, id > 0 ? 31 - __clz(id) : 0)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * HIST_BINS; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

struct Settings {
    int local_windows, local_maxdeg, blocks_per_sm, cap_certify;
    long long certify_after;
    int dual_k;
    long long kick_rounds;
};

static Settings settings_of(const eg_arena *ar) {
    return Settings{ar->local_windows, ar->local_maxdeg, ar->blocks_per_sm, ar->cap_certify, ar->certify_after,
                    ar->dual_k, ar->kick_rounds};
}

static void apply(eg_arena *ar, const Settings &S) {
    ar->local_windows = S.local_windows;
    ar->local_maxdeg = S.local_maxdeg;
    ar->blocks_per_sm = S.blocks_per_sm;
    ar->cap_certify = S.cap_certify;
    ar->certify_after = S.certify_after;
    ar->dual_k = S.dual_k;
    ar->kick_rounds = S.kick_rounds;
}

static int ilog2(double x) { return x <= 1.0 ? 0 : (int)std::lround(std::log2(x)); }

// Coarse class of a bin's share of the vertices: 0 under 1%, 1 under 10%,
// 2 under 50%, 3 otherwise.
static char share_class(unsigned long long c, long long n) {
    const double f = (double)c / (double)std::max(1LL, n);
    return f < 0.01 ? '0' : f < 0.10 ? '1' : f < 0.50 ? '2' : '3';
}

// Signature of one arena and weight map (see the file comment).
static eg_status signature(eg_arena *ar, long long scale, long long shift, int credit_bits, long long count,
                           std::string &key, cudaStream_t s) {
    long long C = 0, wmax = 0;
    eg_status rc = compute_bound(ar, scale, shift, &C, &wmax, s);
    if (rc != EG_OK) return rc;
    unsigned long long *d = nullptr, h[2 * HIST_BINS];
    EG_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(h), s));
    EG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(h), s));
    int sms = 0;
    EG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ar->device));
    k_degree_hist<<<sms * 4, 256, 0, s>>>(ar->d, d);
    EG_CUDA_TRY(cudaGetLastError());
    EG_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaFreeAsync(d, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    std::string out_cls, in_cls;
    for (int b = 0; b < HIST_BINS; ++b) {
        out_cls += share_class(h[b], ar->n);
        in_cls += share_class(h[HIST_BINS + b], ar->n);
    }
    // trailing empty bins carry no information
    while (out_cls.size() > 1 && out_cls.back() == '0') out_cls.pop_back();
    while (in_cls.size() > 1 && in_cls.back() == '0') in_cls.pop_back();
    const int bits = credit_bits != 0 ? credit_bits : (C + wmax <= 0x7fffffffLL - 1 ? 32 : 64);
    char buf[160];
    snprintf(buf, sizeof(buf), "%sn%d-d%d-o%s-i%s-b%d-r%d", count > 1 ? ("plan" + std::to_string(count) + "-").c_str() : "",
             ilog2((double)ar->n), (int)std::lround((double)ar->m / std::max(1, ar->n)), out_cls.c_str(),
             in_cls.c_str(), bits, ilog2((double)C / (double)std::max(1LL, wmax)));
    key = buf;
    return EG_OK;
}

// ---------------------------------------------------------------------------
// The cache file: one JSON object per line with the fields of Settings and
// the key.  Only lines this file writes are read back; others are kept as
// they are when the file is rewritten.

static bool field(const std::string &line, const char *name, long long &v) {
    const std::string pat = std::string("\"") + name + "\":";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    p += pat.size();
    while (p < line.size() && line[p] == ' ') ++p;
    char *end = nullptr;
    v = strtoll(line.c_str() + p, &end, 10);
    return end != line.c_str() + p;
}

static bool key_of(const std::string &line, std::string &key) {
    const std::string pat = "\"key\": \"";
    size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    p += pat.size();
    const size_t q = line.find('"', p);
    if (q == std::string::npos) return false;
    key = line.substr(p, q - p);
    return true;
}

static std::vector<std::string> read_lines(const char *path) {
    std::vector<std::string> lines;
    FILE *fh = fopen(path, "r");
    if (!fh) return lines;
    std::string cur;
    int c;
    while ((c = fgetc(fh)) != EOF) {
        if (c == '\n') {
            if (!cur.empty()) lines.push_back(cur);
            cur.clear();
        } else {
            cur += (char)c;
        }
    }
    if (!cur.empty()) lines.push_back(cur);
    fclose(fh);
    return lines;
}

static bool cache_lookup(const char *path, const std::string &key, Settings &S, double &ms) {
    for (const std::string &line : read_lines(path)) {
        std::string k;
        if (!key_of(line, k) || k != key) continue;
        long long lw, md, bps, cc, ca, dk, kr, us = -1;
        if (field(line, "local_windows", lw) && field(line, "local_maxdeg", md) && field(line, "blocks_per_sm", bps) &&
            field(line, "cap_certify", cc) && field(line, "certify_after", ca) && field(line, "dual_k", dk) &&
            field(line, "kick_rounds", kr)) {
            field(line, "tuned_us", us);
            S = Settings{(int)lw, (int)md, (int)bps, (int)cc, ca, (int)dk, kr};
            ms = us >= 0 ? us * 1e-3 : -1.0;
            return true;
        }
    }
    return false;
}

static eg_status cache_store(const char *path, const std::string &key, const Settings &S, double ms) {
    std::vector<std::string> keep;
    for (const std::string &line : read_lines(path)) {
        std::string k;
        if (key_of(line, k) && k == key) continue;
        keep.push_back(line);
    }
    char buf[512];
    snprintf(buf, sizeof(buf),
             "{\"key\": \"%s\", \"local_windows\": %d, \"local_maxdeg\": %d, \"blocks_per_sm\": %d, "
             "\"cap_certify\": %d, \"certify_after\": %lld, \"dual_k\": %d, \"kick_rounds\": %lld, "
             "\"tuned_us\": %lld}",
             key.c_str(), S.local_windows, S.local_maxdeg, S.blocks_per_sm, S.cap_certify, S.certify_after,
             S.dual_k, S.kick_rounds, (long long)std::llround(ms * 1e3));
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fh = fopen(tmp.c_str(), "w");
    if (!fh) {
        set_error("cannot write the tuning cache %s", tmp.c_str());
        return EG_ERR_INVALID;
    }
    for (const std::string &line : keep) fprintf(fh, "%s\n", line.c_str());
    if (fclose(fh) != 0 || rename(tmp.c_str(), path) != 0) {
        set_error("cannot replace the tuning cache %s", path);
        return EG_ERR_INVALID;
    }
    return EG_OK;
}

// ---------------------------------------------------------------------------
// The search.

// One timed run of the instance with the arena's current settings: device
// time from an event before to an event after it on s; negative on failure.
typedef eg_status (*RunFn)(void *ctx, cudaStream_t s);

static eg_status timed(RunFn run, void *ctx, cudaStream_t s, int reps, double &ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EG_CUDA_TRY(cudaEventCreate(&e0));
    EG_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<double> t;
    eg_status rc = EG_OK;
    for (int k = 0; k < reps && rc == EG_OK; ++k) {
        cudaEventRecord(e0, s);
        rc = run(ctx, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != EG_OK) return rc;
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return EG_OK;
}

// Coordinate search from the arena's settings: each setting in turn takes
// the value of its candidate list that times best with the others fixed.
// A candidate replaces the best only if more than 3% faster.  Stops after
// max_solves timed runs.
static eg_status search(eg_arena *ar, RunFn run, void *ctx, cudaStream_t s, int max_solves, bool trials_matter,
                        double &default_ms, double &best_ms, int &solves) {
    // the first run warms the caches of launch settings and scratch
    double warm = 0;
    eg_status rc = timed(run, ctx, s, 1, warm);
    if (rc != EG_OK) return rc;
    const int reps = warm < 20.0 ? 5 : warm < 200.0 ? 3 : 1;
    rc = timed(run, ctx, s, reps, default_ms);
    if (rc != EG_OK) return rc;
    solves = 1 + reps;
    best_ms = default_ms;
    Settings best = settings_of(ar);
    const int lw[] = {0, 16, 32, 64, 128, 256};
    const int md[] = {8, 16, 32, 64, 256};
    const int bps[] = {1, 2, 3, 0};
    const int cc[] = {2, 4, 8, 16};
    const int dk[] = {1, 2, 4, 8};
    const int ca[] = {0, 4, 8, 16, 32};
    const int kr[] = {0, 1, 2, 4, 8};
    // the route's settings first (the first attempt, the jumps' slices, the
    // trials' cap and K): they change the work most
    const int order[] = {4, 6, 3, 5, 0, 1, 2};
    for (int dim : order) {
        if ((dim == 3 || dim == 4 || dim == 5 || dim == 6) && !trials_matter) continue;
        const int *vals = dim == 0   ? lw
                          : dim == 1 ? md
                          : dim == 2 ? bps
                          : dim == 3 ? cc
                          : dim == 5 ? dk
                          : dim == 6 ? kr
                                     : ca;
        const int nv = dim == 0 ? 6 : (dim == 1 || dim == 4 || dim == 6) ? 5 : 4;
        for (int k = 0; k < nv; ++k) {
            if (solves + reps > max_solves) break;
            Settings c = best;
            int *slot = dim == 0 ? &c.local_windows : dim == 1 ? &c.local_maxdeg : dim == 2 ? &c.blocks_per_sm
                                                      : dim == 5 ? &c.dual_k : &c.cap_certify;
            if (dim == 4 || dim == 6) {
                long long &v = dim == 4 ? c.certify_after : c.kick_rounds;
                if (v == vals[k]) continue;
                v = vals[k];
            } else {
                if (*slot == vals[k]) continue;
                *slot = vals[k];
            }
            apply(ar, c);
            double ms = 0;
            rc = timed(run, ctx, s, reps, ms);
            solves += reps;
            if (rc != EG_OK) {
                apply(ar, best);
                return rc;
            }
            if (ms < best_ms * 0.97) {
                best_ms = ms;
                best = c;
            }
        }
    }
    apply(ar, best);
    return EG_OK;
}

struct SingleCtx {
    eg_arena *ar;
    int bits;
    long long scale, shift;
    void *out;
};

static eg_status run_single(void *p, cudaStream_t s) {
    SingleCtx *c = (SingleCtx *)p;
    return solve(c->ar, c->bits, c->scale, c->shift, c->out, nullptr, s, 0);
}

struct PlanCtx {
    eg_plan_impl *plan;
    void *out;
};

static eg_status run_plan(void *p, cudaStream_t s) {
    PlanCtx *c = (PlanCtx *)p;
    return plan_run(c->plan, c->out, nullptr, s, 0);
}

static void fill(eg_tuning *out, const Settings &S, double d, double t, int solves, int cached, const std::string &key) {
    if (!out) return;
    out->local_windows = S.local_windows;
    out->local_maxdeg = S.local_maxdeg;
    out->blocks_per_sm = S.blocks_per_sm;
    out->cap_certify = S.cap_certify;
    out->certify_after = S.certify_after;
    out->dual_k = S.dual_k;
    out->kick_rounds = (int32_t)S.kick_rounds;
    out->default_ms = d;
    out->tuned_ms = t;
    out->solves = solves;
    out->from_cache = cached;
    snprintf(out->key, sizeof(out->key), "%s", key.c_str());
}

// The shared part of both entry points: signature, cache, search, store.
static eg_status tune(eg_arena *ar, const std::string &key, RunFn run, void *ctx, bool trials_matter,
                      const char *cache_path, int max_solves, eg_tuning *out, cudaStream_t s) {
    Settings S{};
    double ms = -1;
    if (cache_path && cache_lookup(cache_path, key, S, ms)) {
        apply(ar, S);
        fill(out, S, -1.0, ms, 0, 1, key);
        return EG_OK;
    }
    double d = 0, t = 0;
    int solves = 0;
    eg_status rc = search(ar, run, ctx, s, max_solves > 0 ? max_solves : 60, trials_matter, d, t, solves);
    if (rc != EG_OK) return rc;
    S = settings_of(ar);
    if (cache_path && (rc = cache_store(cache_path, key, S, t)) != EG_OK) return rc;
    fill(out, S, d, t, solves, 0, key);
    return EG_OK;
}

}  // namespace eg

extern "C" {

eg_status eg_autotune(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift, const char *cache_path,
                      int32_t max_solves, eg_tuning *out) {
    eg::clear_error();
    if (!arena || (credit_bits != 0 && credit_bits != 32 && credit_bits != 64) || max_solves < 0) {
        eg::set_error("need an arena, credit_bits 0/32/64 and max_solves >= 0");
        return EG_ERR_INVALID;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        eg::set_error("stream creation failed");
        return EG_ERR_CUDA;
    }
    void *buf = nullptr;
    eg_status rc = EG_OK;
    std::string key;
    if (cudaMalloc(&buf, (size_t)arena->n * 8) != cudaSuccess) {
        cudaGetLastError();
        eg::set_error("device buffer for the timed solves failed");
        rc = EG_ERR_OOM;
    }
    if (rc == EG_OK) rc = eg::signature(arena, w_scale, w_shift, credit_bits, 1, key, s);
    if (rc == EG_OK) {
        // a first solve tells whether the certified trials run at all
        eg_stats st{};
        rc = eg::solve(arena, credit_bits, w_scale, w_shift, buf, &st, s, 0);
        if (rc == EG_OK) {
            eg::SingleCtx ctx{arena, credit_bits, w_scale, w_shift, buf};
            rc = eg::tune(arena, key, eg::run_single, &ctx, st.trials > 0, cache_path, max_solves, out, s);
        }
    }
    if (buf) cudaFree(buf);
    cudaStreamDestroy(s);
    return rc;
}

eg_status eg_plan_autotune(eg_plan *plan, const char *cache_path, int32_t max_solves, eg_tuning *out) {
    eg::clear_error();
    eg::eg_plan_impl *p = eg::plan_impl(plan);
    if (!p || max_solves < 0) {
        eg::set_error("need a plan and max_solves >= 0");
        return EG_ERR_INVALID;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        eg::set_error("stream creation failed");
        return EG_ERR_CUDA;
    }
    long long total = 0;
    for (int i = 0; i < eg::plan_count(p); ++i) {
        long long n = 0;
        eg::plan_instance_info(p, i, nullptr, &n, nullptr, nullptr);
        total += n;
    }
    void *buf = nullptr;
    eg_status rc = EG_OK;
    std::string key;
    if (cudaMalloc(&buf, (size_t)total * 8) != cudaSuccess) {
        cudaGetLastError();
        eg::set_error("device buffer for the timed runs failed");
        rc = EG_ERR_OOM;
    }
    eg_arena *ar = p ? eg::plan_arena(p) : nullptr;
    if (rc == EG_OK) rc = eg::signature(ar, 1, 0, eg::plan_bits(p), eg::plan_count(p), key, s);
    if (rc == EG_OK) {
        eg_stats st{};
        rc = eg::plan_run(p, buf, &st, s, 0);
        if (rc == EG_OK) {
            eg::PlanCtx ctx{p, buf};
            rc = eg::tune(ar, key, eg::run_plan, &ctx, st.trials > 0, cache_path, max_solves, out, s);
        }
    }
    if (buf) cudaFree(buf);
    cudaStreamDestroy(s);
    return rc;
}

}  // extern "C"
