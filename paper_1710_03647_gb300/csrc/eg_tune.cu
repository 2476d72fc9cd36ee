// Autotuner of the solver's launch settings (eg_autotune, eg_plan_autotune),
// with a cache of chosen settings on disk.
//
// The settings that change how fast the least fixpoint is reached -- never
// the result -- are the per-warp local worklist budget and its degree
// threshold, the resident blocks per SM of the persistent kernel, the dense
// sweeps before the worklist rounds, the chunk size of long worklists, and
// the certified route's first trial cap, dual K, cycle-jump slice length and
// the round budget of its first attempt.  The best values depend on the arena: R-MAT's power-law rows
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
    long long v[9];  // the values of the tuned options, in the order of DIMS
};

// The options the search tunes, with their candidate values.  `trials`:
// the option only matters where the certified trials run.
struct Dim {
    const char *name;  // the field's name in the cache file
    bool trials;
    int nvals;
    long long vals[6];
};
static const Dim DIMS[9] = {
    {"local_windows", false, 6, {0, 16, 32, 64, 128, 256}},
    {"local_maxdeg", false, 5, {8, 16, 32, 64, 256}},
    {"blocks_per_sm", false, 4, {1, 2, 3, 0}},
    {"cap_certify", true, 4, {2, 4, 8, 16}},
    {"certify_after", true, 5, {0, 4, 8, 16, 32}},
    {"dual_k", true, 4, {1, 2, 4, 8}},
    {"kick_rounds", true, 5, {0, 1, 2, 4, 8}},
    {"sweeps", false, 5, {0, 1, 2, 4, 8}},
    {"chunk_edges", false, 5, {0, 512, 1024, 2048, 4096}},
};
enum { D_LW, D_MD, D_BPS, D_CC, D_CA, D_DK, D_KR, D_SW, D_CH };

static Settings settings_of(const eg_arena *ar) {
    Settings S;
    S.v[D_LW] = ar->local_windows;
    S.v[D_MD] = ar->local_maxdeg;
    S.v[D_BPS] = ar->blocks_per_sm;
    S.v[D_CC] = ar->cap_certify;
    S.v[D_CA] = ar->certify_after;
    S.v[D_DK] = ar->dual_k;
    S.v[D_KR] = ar->kick_rounds;
    S.v[D_SW] = ar->sweeps;
    S.v[D_CH] = ar->chunk_edges;
    return S;
}

static void apply(eg_arena *ar, const Settings &S) {
    ar->local_windows = (int)S.v[D_LW];
    ar->local_maxdeg = (int)S.v[D_MD];
    ar->blocks_per_sm = (int)S.v[D_BPS];
    ar->cap_certify = (int)S.v[D_CC];
    ar->certify_after = S.v[D_CA];
    ar->dual_k = (int)S.v[D_DK];
    ar->kick_rounds = S.v[D_KR];
    ar->sweeps = (int)S.v[D_SW];
    ar->chunk_edges = (int)S.v[D_CH];
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
        Settings c;
        bool all = true;
        for (int d = 0; d < 9 && all; ++d) all = field(line, DIMS[d].name, c.v[d]);
        if (!all) continue;  // a line of an older field set: not a hit
        long long us = -1;
        field(line, "tuned_us", us);
        S = c;
        ms = us >= 0 ? us * 1e-3 : -1.0;
        return true;
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
    std::string rec = "{\"key\": \"" + key + "\"";
    for (int d = 0; d < 9; ++d) rec += std::string(", \"") + DIMS[d].name + "\": " + std::to_string(S.v[d]);
    rec += ", \"tuned_us\": " + std::to_string((long long)std::llround(ms * 1e3)) + "}";
    keep.push_back(rec);
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
    // the settings that change the work most first: the first attempt's
    // budget, the sweeps, the local worklist budget, then the trials' jump
    // slices, cap and K
    const int order[] = {D_CA, D_SW, D_LW, D_KR, D_CC, D_DK, D_CH, D_MD, D_BPS};
    for (int d : order) {
        if (DIMS[d].trials && !trials_matter) continue;
        for (int k = 0; k < DIMS[d].nvals; ++k) {
            if (solves + reps > max_solves) break;
            Settings c = best;
            if (c.v[d] == DIMS[d].vals[k]) continue;
            c.v[d] = DIMS[d].vals[k];
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
    out->local_windows = (int32_t)S.v[D_LW];
    out->local_maxdeg = (int32_t)S.v[D_MD];
    out->blocks_per_sm = (int32_t)S.v[D_BPS];
    out->cap_certify = (int32_t)S.v[D_CC];
    out->certify_after = S.v[D_CA];
    out->dual_k = (int32_t)S.v[D_DK];
    out->kick_rounds = (int32_t)S.v[D_KR];
    out->sweeps = (int32_t)S.v[D_SW];
    out->chunk_edges = (int32_t)S.v[D_CH];
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
