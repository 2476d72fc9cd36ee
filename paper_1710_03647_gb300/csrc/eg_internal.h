// Internal definitions shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/eg.h"

namespace eg {

// Thread-local message behind eg_last_error().
void set_error(const char *fmt, ...);
void clear_error();

#define EG_CUDA_TRY(expr)                                                                    \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess) {                                                             \
            ::eg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                            __LINE__);                                                       \
            return _e == cudaErrorMemoryAllocation ? EG_ERR_OOM : EG_ERR_CUDA;               \
        }                                                                                    \
    } while (0)

// Control block of one solve, in device memory.  Lists for round r live in
// buffer r & 1; their packed counters in slot r % 3 (low 32 bits: entries,
// high 32 bits: total work = edges to scan).
struct Ctrl {
    unsigned long long pull_ctr[3];
    unsigned long long push_ctr[3];
    unsigned int bar_count;
    unsigned int bar_gen;
    int status;
    unsigned stop_flag;  // a slice of a resident solve ends after this round (doorbell seen)
    unsigned long long rounds, lifts, pushes, relax, enqueues, seeded;
    long long r_next;    // round a resident solve resumes at
    unsigned pull_take[3], push_take[3];  // chunks of round r's lists taken so far (slot r % 3)
};

// Read-only arena data on the device (int32 offsets: m < 2^31).
struct DevArena {
    int n;
    int m;
    const int *row_ptr;         // n + 1
    const int *col;             // m
    const int *w;               // m
    const int *rrow_ptr;        // n + 1
    const unsigned *rcol;       // m: predecessor id | (owner(pred) is V1) << 31
    const int *rw;              // m: w(pred, v)
    const unsigned *owner_bits; // ceil(n / 32)
    const int *wmin;            // n: smallest weight on the vertex's out-edges
    const int *wmax;            // n: largest weight on the vertex's out-edges
};

// Weight view w' = scale * w - shift and the bound C of that view.
struct WeightView {
    long long scale;
    long long shift;
    long long C;
};

// Mutable per-solve state for one credit width.
struct DevState {
    void *f;           // int32 or int64 credits, n
    int *pull_items[2];
    int *pull_offs[2];
    int *push_items[2];
    int *push_offs[2];
    unsigned *bits_pull[2]; // dedupe bitmaps of the pull lists, ceil(n/32) words
    unsigned *bits_push[2]; // dedupe bitmaps of the push lists
    unsigned *seed_bits;    // warm-start marks, ceil(n/32) words
    void *acc;         // partial minima of split player-0 lifts, n (TOP when idle)
    int *acc_done;     // edges accounted into acc, n (0 when idle)
    Ctrl *ctrl;
};

struct StateBuffers {
    int bits = 0;      // 0 = not allocated, else 32 / 64
    long long nf = 0;  // credits the buffers hold
    bool dirty = true; // scratch (acc, acc_done, bitmaps) needs resetting
    DevState d{};
    void *block = nullptr;
    size_t bytes = 0;
};

}  // namespace eg

struct eg_arena {
    int device = 0;
    int n = 0;
    int m = 0;
    void *block = nullptr;  // one allocation holding the read-only arrays
    eg::DevArena d{};
    long long C_plain = -1, wmax_plain = -1;  // bound and max |w| for scale 1, shift 0
    eg::StateBuffers st32, st64;
    eg::StateBuffers st_dual;  // int64 state of the certified trials' dual lifts
    eg::StateBuffers st_dual32;  // int32 state of the dual lifts whose cap and weights fit int32
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk = nullptr;
    void *host_ctrl = nullptr;  // pinned copy of Ctrl
    int local_windows = 64;     // per-warp local worklist budget per round (0 disables chaining)
    int local_maxdeg = 64;      // largest degree of a vertex handled through the local worklist
    int chunk_edges = 1024;     // edges per chunk of a round's list that spans more per warp (0: one chunk per warp)
    int sweeps = 0;             // dense sweeps (in-place lifts of every credit) before the worklist rounds
    int warm_start = 1;         // TOP on player-1 negative cycles of length <= 2 before lifting
    long long seed_max_pairs = 4096;
    int use_graph = 1;                // batched solves replay a captured graph
    int cap_certify = 4;              // first trial cap of the certified solve, in units of max|w'| (0: off)
    int dual_k = 4;                   // weight multiplier K of the first trial's dual lift
    long long kick_rounds = 2;        // rounds between cycle jumps of the trials' lifts (0: none)
    void *kick_block = nullptr;       // scratch of the cycle jumps (allocated on first use)
    unsigned kick_epoch = 0;          // epoch counter of its claim array
    long long certify_after = 64;     // rounds of a first solve with cap C before the trial caps (0: none); eg_create sets the default
    int blocks_per_sm = 0;            // resident blocks per SM of the fixpoint kernel (0: as many as fit)
    int scc_order = 0;                // solve by the topological levels of the strongly connected components
    int *scc_level = nullptr;         // condensation (computed on first use): level of each vertex,
    int *scc_comp = nullptr;          //   representative of its component,
    int scc_nlevels = 0, scc_count = 0, scc_passes = 0;  //   levels, components, kernel passes taken
    unsigned long long wait_limit_ns = 5000000000ull;  // limit of each grid-barrier wait
    void *cert_block = nullptr;       // device memory of the certified solve:
    unsigned long long *aux = nullptr;  //   counters (4 words)
    unsigned *cert_w0 = nullptr;      //   bitmap of vertices proven won by player 0
    unsigned *cert_w1 = nullptr;      //   bitmap of vertices proven won by player 1
    std::vector<long long> part_ptr;  // game boundaries (empty: one game)
};

namespace eg {
// Implemented in eg_solve.cu
eg_status compute_bound(eg_arena *a, long long scale, long long shift, long long *C, long long *wmax,
                        cudaStream_t s);
// eg_solve_credit's route; with attempt_only > 0 only its first attempt (cap
// C, that many rounds), which ends with EG_ERR_BUDGET if it does not finish.
eg_status solve(eg_arena *a, int credit_bits, long long scale, long long shift, void *out, eg_stats *st,
                cudaStream_t s, long long max_rounds, long long attempt_only = 0);
eg_status free_state(StateBuffers &sb);
// The strongly connected components and their topological levels (eg_scc.cu),
// computed once per arena.
eg_status scc_levels(eg_arena *a, cudaStream_t s);

// Resident solve (eg_solve.cu), used by the server: one int64 solve state
// over a pool of `cap` credits that holds up to `slots` games at a time.
// Games join at a round boundary (resident_admit: weight view, warm start
// and initial push list of the game's credit range) while others are
// mid-solve; resident_slice runs the persistent fixpoint from the current
// round until the doorbell rings, `rounds` rounds pass or no work is left;
// resident_busy marks the slots that still have queued work, so the others
// are finished.  The owner keeps A (the pool arena) valid for every range it
// admits.
struct Resident {
    int device = 0;
    int cap = 0;
    int slots = 0;
    DevArena A{};
    StateBuffers sb;
    void *block = nullptr;     // inst_id[cap], busy[slots], delta[slots], scale/shift/C[slots]
    int *inst_id = nullptr;
    int *busy = nullptr;
    int *delta = nullptr;
    long long *scale = nullptr, *shift = nullptr, *C = nullptr;
    unsigned *bell_host = nullptr;  // mapped pinned flag; non-zero ends the running slice
    unsigned *bell_dev = nullptr;
    void *host_ctrl = nullptr;      // pinned copy of the control block after a slice
    int *host_busy = nullptr;       // pinned copy of busy
    long long *host_tab = nullptr;  // pinned staging of the slot tables (scale, shift, C per slot)
    long long r = 0;                // next round
    int local_windows = 64, local_maxdeg = 64;
    int chunk_edges = 1024;  // edges per chunk of a long list (0: one chunk per warp)
    long long seed_max_pairs = 4096;
};
eg_status resident_create(Resident &R, int device, int cap, int slots, cudaStream_t s);
void resident_free(Resident &R);
eg_status resident_reset(Resident &R, cudaStream_t s);
eg_status resident_admit(Resident &R, int slot, int g0, int n, long long scale, long long shift, long long C,
                         cudaStream_t s);
eg_status resident_slice(Resident &R, long long rounds, cudaStream_t s, int *dev_status);
eg_status resident_busy(Resident &R, cudaStream_t s);

// Batched solves (eg_solve.cu), used by the server.
struct eg_plan_impl;
eg_status plan_create(eg_arena *ar, int count, const int32_t *part, const int64_t *w_scale, const int64_t *w_shift,
                      int credit_bits, eg_plan_impl **out);
eg_status plan_run(eg_plan_impl *p, void *out, eg_stats *st, cudaStream_t user, long long max_rounds);
eg_status plan_release(eg_plan_impl *p);
void plan_instance_info(const eg_plan_impl *p, int i, long long *offset, long long *n, long long *C, int *bits);
eg_plan_impl *plan_impl(eg_plan *plan);
eg_arena *plan_arena(const eg_plan_impl *p);
int plan_count(const eg_plan_impl *p);
int plan_bits(const eg_plan_impl *p);  // the width the plan computes in
}  // namespace eg
