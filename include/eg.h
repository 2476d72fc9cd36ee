/*
 * eg.h -- C ABI of the GB300 energy-game solver.
 *
 * Problem (arXiv 1710.03647, Sec. 3, Def. "Initial Credit Problem"): for a
 * total weighted game arena G = (V, E, w, <V0, V1>) (Sec. 2), decide for every
 * vertex v whether player 0 wins the energy objective (Eq. 1) and, if so,
 * the minimum initial credit c(v).  The solver computes the least energy
 * progress measure (Def. "EPM", Sec. 3.1) as the least fixpoint of the
 * lifting operator (Def. "Lifting Operator") with the bounded operator
 * a (-) b = TOP if a = TOP or a - b > C, else max(0, a - b), where C = M_G,
 * the bound of Sec. 3.1.  TOP marks the vertices player 1 wins.
 *
 * Conventions for every call:
 *   - No exception or C++ type crosses this boundary; every call returns an
 *     eg_status, and on failure eg_last_error() gives a message for the
 *     calling thread.
 *   - Vertex ids are 0..n-1 in the caller's order; results use that order.
 *   - Ownership is a bitmap of ceil(n/32) uint32 words: bit (v % 32) of word
 *     v / 32 is 1 iff v is a player-1 vertex (V1), 0 iff player 0 (V0).
 *   - Weights are int32.  A solve may view them through the integer map
 *     w' = w_scale * w - w_shift (a mean-payoff threshold query, Sec. 3 on
 *     the reduction between energy and mean-payoff games); the map is
 *     applied on the fly, the arena is not rewritten.
 *   - Host pointers are plain host memory; "device" pointers are CUDA device
 *     memory of the current device.
 */
#ifndef EG_H
#define EG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t eg_status;
#define EG_OK 0
#define EG_PENDING 1           /* eg_poll: request not finished yet */
#define EG_ERR_INVALID (-1)    /* malformed arguments or CSR arrays */
#define EG_ERR_NOT_TOTAL (-2)  /* a vertex has no successor (Sec. 2 assumes totality) */
#define EG_ERR_OVERFLOW (-3)   /* int32 credits asked for but C + max|w'| does not fit */
#define EG_ERR_OOM (-4)        /* device or host allocation failed */
#define EG_ERR_CUDA (-5)       /* a CUDA runtime call failed */
#define EG_ERR_TIMEOUT (-6)    /* a device-side wait ran past its spin limit */
#define EG_ERR_BUDGET (-7)     /* the round budget ran out before the fixpoint */
#define EG_ERR_BUSY (-8)       /* the server cannot take more requests now */

#define EG_TOP32 INT32_MAX     /* TOP in int32 credit arrays */
#define EG_TOP64 INT64_MAX     /* TOP in int64 credit arrays */

/* eg_create flags */
#define EG_INPUT_DEVICE 1u     /* the CSR/bitmap pointers are device pointers */

typedef struct eg_arena eg_arena;
typedef struct eg_server eg_server;

#define EG_MAX_PHASES 16
#define EG_PHASE_ATTEMPT 0     /* lift with cap C under a round budget (or the only lift) */
#define EG_PHASE_DUAL 1        /* certified trial: lift of the dual game */
#define EG_PHASE_CAPPED 2      /* certified trial: lift of the game with cap B */
#define EG_PHASE_FINAL 3       /* lift with cap C from the trials' proven TOP starts */
#define EG_PHASE_LEVEL 4       /* SCC-ordered solve: lift of one topological level */

/* Counters of one solve.  relaxations counts evaluations of f(u) (-) w over
 * edges (pulls of player-0 lifts plus pushes to predecessors); lifts counts
 * player-0 vertices lifted; pushes counts vertices whose rise was sent to
 * their predecessors; rounds counts frontier rounds (Algorithm 3's loop). */
typedef struct eg_stats {
    int64_t C;             /* the bound M_G of the (mapped) weights */
    int64_t seeded;        /* vertices the warm start set to TOP (0 without it) */
    int32_t credit_bits;   /* width the solve computed in: 32 or 64 */
    int32_t status;        /* the solve's eg_status */
    int64_t rounds;
    int64_t lifts;
    int64_t pushes;
    int64_t relaxations;
    int64_t enqueues;
    double ms;             /* device time of initialisation + fixpoint kernels */
    double fixpoint_ms;    /* device time of the lifting kernels alone: the dense sweeps
                            * (EG_OPT_SWEEPS) and the persistent fixpoint kernel */
    int64_t cycle_jumps;   /* vertices raised by cycle jumps (EG_OPT_KICK_ROUNDS) */
    /* The fixpoint launches of the solve in order, the first EG_MAX_PHASES
     * of them: a single solve runs a first attempt with cap C and, when that
     * does not finish, certified trials (a dual lift and a capped lift each,
     * see EG_OPT_CAP_CERTIFY) and possibly a final lift with cap C. */
    int32_t phases;        /* launches recorded below */
    int32_t trials;        /* certified trials run (0: the first attempt finished) */
    int32_t phase_kind[EG_MAX_PHASES];        /* EG_PHASE_* */
    int64_t phase_cap[EG_MAX_PHASES];         /* the launch's cap: C, (K + 1) B or B */
    int64_t phase_rounds[EG_MAX_PHASES];
    int64_t phase_relaxations[EG_MAX_PHASES];
    double phase_ms[EG_MAX_PHASES];           /* device time of its sweeps and fixpoint kernel */
} eg_stats;

/*
 * eg_create -- copy an arena to the device and build what the solver needs.
 *
 * Arena of Sec. 2: n vertices, m edges in forward CSR
 *   row_ptr[n+1] (int64, row_ptr[0] = 0, non-decreasing, row_ptr[n] = m),
 *   col[m] (int32 successor ids), w[m] (int32 weights w(v, col)).
 * The predecessor sets pre(v) (Sec. 2) come as the reverse CSR
 *   rrow_ptr[n+1], rcol[m] (predecessor ids), rw[m] (w of that edge),
 * or all three NULL, in which case the library builds them on the device.
 * A given reverse CSR must hold exactly the edges of the forward one (checked
 * with a multiset hash; EG_ERR_INVALID otherwise).
 * owner_bits: ceil(n/32) words as above.
 *
 * Requires 1 <= n < 2^31 and n <= m < 2^31.  Every vertex must have a
 * successor (EG_ERR_NOT_TOTAL otherwise).  Duplicate edges and self-loops
 * are allowed.  flags: EG_INPUT_DEVICE or 0 (host inputs).
 *
 * Ownership: the inputs stay the caller's and are not referenced after the
 * call returns; the returned arena (and all device memory it holds) belongs
 * to the library until eg_destroy.  Synchronous.
 */
eg_status eg_create(int64_t n, int64_t m,
                    const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                    const int64_t *rrow_ptr, const int32_t *rcol, const int32_t *rw,
                    const uint32_t *owner_bits, uint32_t flags, eg_arena **out);

/* eg_destroy -- free an arena and its device memory.  NULL is accepted. */
eg_status eg_destroy(eg_arena *arena);

/*
 * eg_bound -- the bound C = M_G (Sec. 3.1) of the arena under the map
 * w' = w_scale * w - w_shift, and the largest |w'|; either output may be NULL.
 */
eg_status eg_bound(eg_arena *arena, int64_t w_scale, int64_t w_shift, int64_t *C, int64_t *max_abs_w);

/*
 * eg_solve_credit -- the least energy progress measure (Sec. 3.1), i.e. the
 * minimum initial credits with TOP on the player-1 winning set.
 *
 * credit_bits: 32 -> credits_out is int32[n] (TOP = EG_TOP32), and the solve
 *   fails with EG_ERR_OVERFLOW unless C + max|w'| <= INT32_MAX - 1;
 *   64 -> credits_out is int64[n] (TOP = EG_TOP64), computed in int64;
 *   0 -> credits_out is int64[n]; the solve computes in int32 when the rule
 *   above allows it, else in int64.
 * w_scale / w_shift: weight map as above (1 and 0 for the plain arena);
 *   |w_scale| * 2^31 + |w_shift| must stay below 2^62.
 * credits_out: host or device pointer (detected), caller-owned, n elements.
 * st: optional counters (may be NULL).
 * cuda_stream: the cudaStream_t to run on (NULL = the legacy default stream).
 * max_rounds: round budget of each fixpoint launch (0 = unlimited);
 *   EG_ERR_BUDGET when one runs out.
 * Synchronous: returns after the credits are written.  One solve at a time
 * per arena.  EG_ERR_TIMEOUT if a device-side wait gave up (see
 * EG_OPT_WAIT_LIMIT_US); the device stays usable and the arena can be solved
 * again.  After EG_ERR_BUDGET or EG_ERR_TIMEOUT every credit written is at or
 * below the least fixpoint: the values a lift with cap C reached before it
 * stopped, or 0 where the solve stopped inside a certified trial and no such
 * lift had run.
 */
eg_status eg_solve_credit(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                          void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds);

/*
 * eg_strategy -- a winning positional strategy of player 0 read off the
 * least EPM (Def. "EPM", Sec. 3.1; the problem statement of Sec. 3 asks for
 * the credits and the strategies that achieve them).  For every player-0
 * vertex v with a finite credit, succ_out[v] is the successor u of v's first
 * out-edge (in CSR order) with f(u) (-) w'(v, u) = f(v); every other vertex
 * gets -1.  Following it from v, player 0 never needs more than f(v)
 * energy: every cycle of chosen edges has weight >= 0.
 *
 * credits: n credits of credit_bits (32 or 64), as eg_solve_credit wrote
 * them for the same weight map w' = w_scale * w - w_shift; host or device
 * pointer.  succ_out: int32[n], host or device pointer, caller-owned.
 * Synchronous.  EG_ERR_INVALID if a finite player-0 credit is attained by
 * no out-edge (then the credits are not the least EPM of this arena and
 * map).  Allocates scratch of about n * (credit_bits / 8 + 4) bytes on the
 * stream's memory pool.
 */
eg_status eg_strategy(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift, const void *credits,
                      int32_t *succ_out, void *cuda_stream);

/*
 * eg_set_option -- per-arena settings of later solves.  None of them changes
 * a result: they change only how fast the least fixpoint is reached.
 *
 *   EG_OPT_LOCAL_WINDOWS (default 64): per-warp budget, per round, of
 *     32-entry windows worked through the warp's local worklist, which
 *     carries a rise on to the predecessors within the same round; 0 turns
 *     this off (one hop per round, as in Algorithm 3).
 *   EG_OPT_LOCAL_MAXDEG (default 64): largest degree of a vertex handled
 *     through the local worklist.
 *   EG_OPT_WARM_START (default 1): before lifting, set f = TOP on player-1
 *     vertices that lie on a negative cycle of player-1 vertices of length
 *     1 or 2 (under the weight map).  Player 1 keeps the play on such a
 *     cycle forever, so these vertices are in W1 (Lemma "EGcycles" and
 *     memoryless determinacy, Sec. 3) and TOP is their least-fixpoint
 *     value: the start stays below the least fixpoint and the result is
 *     unchanged.  0 starts from f = 0 everywhere, as the paper does.
 *   EG_OPT_SEED_MAX_PAIRS (default 4096): the warm start skips a vertex
 *     whose out-degree times in-degree exceeds this.
 *   EG_OPT_GRAPH (default 1): batched solves (eg_plan_run) replay a captured
 *     CUDA graph; 0 launches the kernels directly every run.
 *   EG_OPT_CAP_CERTIFY (default 4; used by eg_solve_credit while
 *     EG_OPT_WARM_START is 1): certified trial caps for games the cap-C
 *     lifting is slow on.  A trial lifts the dual game -- weights
 *     -(K w' + 1), owners swapped, cap (K + 1) B -- then the game itself with
 *     cap B.  A vertex finite in the dual is won by player 1 (player 1 then
 *     keeps every cycle of the play at negative weight), so it starts the
 *     game's lift at TOP; a vertex finite in the game's capped lift is won by
 *     player 0, so it starts the next dual lift at TOP.  Once every vertex is
 *     finite or proven lost, every finite credit is at most B, and a cap at or
 *     above the largest finite credit gives the same least fixpoint as C
 *     (Sec. 3.1): the capped result is exact.  Trial k uses
 *     B = value * max|w'| * 4^k and K = EG_OPT_DUAL_K * 8^k (at most n + 1),
 *     k < 6; if no trial is exact the solve ends with cap C from the proven
 *     TOP starts.
 *     This turns the pseudo-polynomial climb of player-1 vertices to C into
 *     climbs to B.  0 turns it off.  max_rounds bounds each fixpoint launch.
 *     A trial lift whose cap plus max|w| fits int32 computes in int32
 *     whatever the solve's width (not in eg_solve_credit_noalloc).
 *   EG_OPT_CERTIFY_AFTER (default 8): with certification on, a plain solve
 *     (cap C, warm start) runs first with this round budget, and the trials
 *     start only if it does not reach the fixpoint; 0 starts with the trials.
 *     The value changes the time to the fixpoint, never the result.
 *   EG_OPT_DUAL_K (default 4): K of the first trial's dual lift.  A larger K
 *     proves player-1 wins on longer cycles of small weight in the first
 *     trial; a smaller one keeps the dual credits, and so the dual lift's
 *     climbs, short.
 *   EG_OPT_KICK_ROUNDS (default 2): the lifts of the certified trials run
 *     in slices of this many rounds, and between slices the cycles of the
 *     current choices (every vertex's best edge) are jumped: on a cycle of
 *     negative weight the least fixpoint must leave the cycle at a player-0
 *     vertex, at a credit at least that vertex's best other option, so the
 *     cycle's credits can rise at once to the bound this gives instead of
 *     one lap per deficit at a time.  The bound is below the least fixpoint,
 *     so the result is unchanged.  Cycles of up to 32 edges through vertices
 *     of out-degree at most 64 are tried.  0 turns the jumps off.
 *   EG_OPT_BLOCKS_PER_SM (default 0): resident blocks per SM of the
 *     persistent fixpoint kernel; 0 takes as many as fit, a larger value is
 *     clamped to what fits.  Fewer blocks make the grid barrier cheaper and
 *     leave fewer lanes in flight.
 *   EG_OPT_WAIT_LIMIT_US (default 5000000, i.e. 5 s): wall-clock limit of
 *     each wait of a block at the fixpoint kernel's grid barrier, in
 *     microseconds (at least 1).  A wait that runs out ends the solve with
 *     EG_ERR_TIMEOUT; every block leaves the kernel at its next barrier, the
 *     device stays usable and the arena can be solved again.  A very small
 *     limit makes ordinary waits run out; that is how the timeout path is
 *     tested.
 *   EG_OPT_SCC_ORDER (default 0): 1 solves by strongly connected components
 *     (the closing remark of Sec. 6): the components' topological levels
 *     (eg_scc_info) are lifted in turn, lowest first, each with cap C and
 *     the lower levels final, as the paper's lifting does (no certified
 *     trials).  A condensation of a single level (one component, as a
 *     road-like grid has) takes the default route instead.
 *     eg_solve_credit_noalloc ignores the option.
 *   EG_OPT_CHUNK_EDGES (default 1024): a round whose worklist holds more than
 *     this many edges per warp of the fixpoint kernel is worked in chunks of
 *     this many edges that the warps take in list order, so the whole grid
 *     sweeps the list together and the credits its gathers reach stay in L2;
 *     a shorter list is cut into one equal piece per warp.  0 always cuts one
 *     piece per warp.
 *   EG_OPT_SWEEPS (default 0, at most 1024): dense sweeps before the
 *     worklist rounds of each fixpoint launch (not the levels of an
 *     SCC-ordered solve).  A sweep raises every credit, in index order and in
 *     place, to its lift over all its edges -- coalesced reads, no atomics --
 *     and the last sweep's raised credits start the worklist rounds.  Lifts
 *     from below stay below the least fixpoint, so the result is unchanged;
 *     sweeps pay off where the first rounds touch most edges anyway.  Their
 *     edge evaluations count in the relaxations; they are not rounds and
 *     max_rounds does not bound them.
 *
 * EG_ERR_INVALID for an unknown option or a value out of range.
 */
#define EG_OPT_LOCAL_WINDOWS 1
#define EG_OPT_LOCAL_MAXDEG 2
#define EG_OPT_WARM_START 3
#define EG_OPT_SEED_MAX_PAIRS 4
#define EG_OPT_GRAPH 5
#define EG_OPT_CAP_CERTIFY 6
#define EG_OPT_CERTIFY_AFTER 7
#define EG_OPT_BLOCKS_PER_SM 8
#define EG_OPT_WAIT_LIMIT_US 9
#define EG_OPT_SCC_ORDER 10
#define EG_OPT_DUAL_K 11
#define EG_OPT_KICK_ROUNDS 12
#define EG_OPT_CHUNK_EDGES 13
#define EG_OPT_SWEEPS 14
eg_status eg_set_option(eg_arena *arena, int32_t option, int64_t value);

/*
 * eg_scc_info / eg_scc_levels -- the strongly connected components of the
 * arena's graph (Sec. 2) and their topological levels: a component from which
 * no edge leaves has level 0, any other one more than the highest level its
 * edges reach, so a vertex's least-EPM value depends only on vertices of its
 * level or lower.  Computed on the device on first use (trimming, max-label
 * colouring, backward closure; Kahn's rounds for the levels, of which at
 * most 4096 are kept: components beyond share the last one) and kept with
 * the arena.  eg_scc_info gives the number of components, of levels and of
 * kernel passes the computation took (any pointer may be NULL);
 * eg_scc_levels copies the level and the component (named by its largest
 * vertex id) of every vertex to int32[n] host or device arrays (either may
 * be NULL).  Both allocate device memory on first use and are synchronous.
 */
eg_status eg_scc_info(eg_arena *arena, int64_t *components, int64_t *levels, int64_t *passes);
eg_status eg_scc_levels(eg_arena *arena, int32_t *level_out, int32_t *component_out);

/*
 * eg_set_parts -- declare the arena a disjoint union of `parts` games: game k
 * owns vertices [part_ptr[k], part_ptr[k+1]) (host array of parts + 1
 * offsets, part_ptr[0] = 0, non-decreasing, part_ptr[parts] = n, no empty
 * part).  Every edge must stay inside its game (EG_ERR_INVALID otherwise).
 * Used by batched solves (eg_plan_create); a plain arena is one part.
 */
eg_status eg_set_parts(eg_arena *arena, int32_t parts, const int64_t *part_ptr);

/*
 * Batched solves.  A plan solves `count` instances in one persistent launch:
 * instance i is game part[i] of the arena (or game i if part is NULL) under
 * the weight map w' = w_scale[i] * w - w_shift[i] (1 and 0 if the arrays
 * are NULL).  Instances may repeat a game -- many mean-payoff threshold
 * queries on one arena (Sec. 3, energy / mean-payoff reduction) keep one
 * copy of the arena and one credit array per query.  Each instance gets its
 * own bound C (Sec. 3.1) and its own credit range; the result of every
 * instance equals eg_solve_credit on that game and map alone.
 *
 * credit_bits: 32 -> int32 credits out (EG_ERR_OVERFLOW unless every
 * instance fits, see eg_solve_credit); 64 or 0 -> int64 out.  The plan
 * computes in int32 when every instance fits and credit_bits != 64.
 * eg_plan_create computes the bounds and allocates the solve state
 * (synchronous).  eg_plan_run replays the solve -- warm start, init and the
 * fixpoint kernel, captured once as a CUDA graph -- and writes instance i's
 * credits at element offset i_off (eg_plan_instance) of credits_out (host
 * or device, caller-owned, total elements = sum of the instances' n).
 * Synchronous; one run at a time per plan; the arena must outlive the plan.
 * max_rounds bounds each fixpoint launch; after EG_ERR_BUDGET or
 * EG_ERR_TIMEOUT every credit written is at or below its instance's least
 * fixpoint (0 where the run stopped inside a certified trial).
 */
typedef struct eg_plan eg_plan;
eg_status eg_plan_create(eg_arena *arena, int32_t count, const int32_t *part, const int64_t *w_scale,
                         const int64_t *w_shift, int32_t credit_bits, eg_plan **out);
/* offset (elements), n, C and the width (32/64) the instance alone would need; any may be NULL */
eg_status eg_plan_instance(eg_plan *plan, int32_t i, int64_t *offset, int64_t *n, int64_t *C, int32_t *bits);
eg_status eg_plan_run(eg_plan *plan, void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds);
eg_status eg_plan_destroy(eg_plan *plan);

/*
 * eg_solve_credit_noalloc -- eg_solve_credit for callers that cannot
 * allocate device memory at solve time: a program whose framework has
 * already handed the GPU's memory to its own caching allocator, or a
 * latency-bound loop where cudaMalloc / cudaFree would synchronise the
 * device and stall other streams.  The paper has no counterpart; it is a
 * deployment variant of the same solve: the same route (a first attempt with
 * cap C and the EG_OPT_CERTIFY_AFTER round budget, then certified trial
 * caps, see EG_OPT_CAP_CERTIFY), the same options and the same results.
 *
 * It allocates nothing: its working memory is one fixed device array inside
 * the library of about 14.9 MB (held by every GPU that loads the library
 * until the process exits), and credits_out -- device memory on the arena's
 * device, n elements of credit_bits (32 or 64 only), aligned to its element
 * size -- serves as the credit array while the solve runs.  The arena must
 * have at most EG_NOALLOC_MAX_VERTICES vertices and live on the current
 * device (EG_ERR_INVALID with a message otherwise, before any work).
 *
 * The first call on a device (and the first after a device reset) looks the
 * working array up on that device; make that first call before any stream
 * capture.  All calls share the one array and each call clears what it needs
 * before use, so calls whose work overlaps on the GPU (other threads, or
 * other streams without ordering between them) race and give undefined
 * results: order them.  Synchronous, like eg_solve_credit; after
 * EG_ERR_BUDGET / EG_ERR_TIMEOUT every credit in credits_out is at or below
 * the least fixpoint, as for eg_solve_credit.
 */
#define EG_NOALLOC_MAX_VERTICES (1 << 18)
eg_status eg_solve_credit_noalloc(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                                  void *credits_out, eg_stats *st, void *cuda_stream, int64_t max_rounds);

/*
 * Autotuning of the launch settings (no counterpart in the paper, whose
 * closing remarks propose customising the launch configuration from an
 * analysis of the input).  The settings of eg_set_option that change only
 * how fast the least fixpoint is reached -- EG_OPT_LOCAL_WINDOWS,
 * EG_OPT_LOCAL_MAXDEG, EG_OPT_BLOCKS_PER_SM and, when the certified trials
 * run, EG_OPT_CAP_CERTIFY, EG_OPT_DUAL_K, EG_OPT_KICK_ROUNDS and
 * EG_OPT_CERTIFY_AFTER -- are chosen by timing
 * real solves (every one of them exact) in a coordinate search that starts
 * from the arena's current settings; a candidate replaces the best so far
 * only if it is more than 3% faster.  The chosen settings are set on the
 * arena (for eg_plan_autotune, on the plan's arena) and returned.
 *
 * cache_path (may be NULL): a text file of JSON lines, one per signature.
 * The signature (key) of an instance is its log2 vertex count, mean degree,
 * coarse log2 histograms of out- and in-degrees, credit width and
 * log2(C / max|w'|), prefixed by "plan<count>-" for plans.  A signature
 * found in the file takes its settings without timing anything
 * (from_cache = 1); otherwise the search runs and its result is written to
 * the file (replacing the file atomically).
 *
 * max_solves: bound on timed runs (0: 60).  Allocates a device buffer for
 * the timed runs' credits and a private stream; synchronous.  Solves and
 * plan runs of the arena must not run concurrently with it.
 */
typedef struct eg_tuning {
    int32_t local_windows, local_maxdeg, blocks_per_sm, cap_certify;
    int64_t certify_after;
    int32_t dual_k, kick_rounds;
    int32_t sweeps, chunk_edges;
    double default_ms;   /* time to the fixpoint with the settings the search started from (-1: cached) */
    double tuned_ms;     /* with the chosen settings (the cached figure when from_cache) */
    int32_t solves;      /* runs timed by this call */
    int32_t from_cache;  /* 1: the settings came from cache_path */
    char key[96];        /* the signature */
} eg_tuning;
eg_status eg_autotune(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift, const char *cache_path,
                      int32_t max_solves, eg_tuning *out);
eg_status eg_plan_autotune(eg_plan *plan, const char *cache_path, int32_t max_solves, eg_tuning *out);

/*
 * Serving, with continuous batching.  A server owns a scheduler thread, a
 * pool of device memory of about device_mem_budget bytes (taken at
 * eg_server_create: about 35% for vertex slots at 74 bytes each, 65% for
 * edges at 16 bytes each) and one resident solve over that pool that holds up
 * to max_batch games at once.  eg_submit queues a solve of `arena` under the
 * map w' = w_scale * w - w_shift and returns a ticket at once.  The scheduler
 * admits queued requests in arrival order whenever a slot is free and the
 * game (n + 1 vertex slots, m edges) fits the free pool: it copies the arena
 * into the pool and adds the game to the running solve at its next round, so
 * requests that arrive while others are being solved join them on the device
 * instead of waiting for them to finish.  The solve runs in slices of rounds
 * that end early when a request arrives.  After each slice, every game with
 * no work left is finished and leaves, freeing its slot and memory for the
 * queue.  A game still unfinished after its arena's EG_OPT_CERTIFY_AFTER
 * rounds (while its EG_OPT_CAP_CERTIFY is on) is taken out and solved alone
 * by eg_solve_credit's certified route; its slot is freed once the resident
 * solve has dropped its remaining work.  A game of at least 2^19 edges fills
 * the GPU alone and gains nothing from sharing it: it skips the pool and is
 * solved by eg_solve_credit's route between slices (its stats are that
 * solve's).  A request that finds the server idle -- nothing resident and no
 * other request queued -- first gets that route's first attempt alone
 * (EG_OPT_CERTIFY_AFTER rounds, or 8): with the device idle, sharing it
 * gains nothing, and most games finish within it; a game it does not finish
 * joins the pool as above.  The result of every request equals eg_solve_credit on its arena
 * alone (the games are disjoint in the pool; each has its own bound C and
 * weight map).  Results wait in pinned host buffers that the server reuses.
 * Do not solve an arena yourself while a request for it is pending.
 *
 * eg_poll returns EG_PENDING until the request is done, then copies its
 * credits (n elements: int32 if credit_bits is 32, else int64; host or
 * device pointer) and its counters, and forgets the ticket.  In the stats, ms
 * is the request's latency from eg_submit to completion (host clock),
 * fixpoint_ms the device time of the slices it took part in, rounds the
 * rounds it was resident, and the work counters those of the whole resident
 * solve over that time (shared with the other games).  A request whose game
 * can never fit the pool completes with EG_ERR_OOM; a request for int32
 * credits whose bound does not fit completes with EG_ERR_OVERFLOW.  The arena
 * must stay alive until its request is polled.  eg_server_destroy ends the
 * running slice and drops queued and unfinished requests.  All calls are
 * thread-safe.
 */
eg_status eg_server_create(size_t device_mem_budget, int32_t max_batch, eg_server **out);
eg_status eg_submit(eg_server *server, eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                    uint64_t *ticket);
eg_status eg_poll(eg_server *server, uint64_t ticket, void *credits_out, eg_stats *st);
eg_status eg_server_destroy(eg_server *server);

/*
 * eg_server_counters_get -- the server's event counts since it was created:
 * requests submitted, admitted into the pool, solved alone by the single-game
 * route (solo: the games that fill the GPU and the requests the idle route
 * answered; idle_solo counts the latter), taken out of the pool to be solved
 * alone by the certified route (taken_out), completed (any status),
 * admission attempts refused for want of pool room (refused; the request
 * stays queued and is retried after the next slice), and slices of the
 * resident solve run.
 */
typedef struct eg_server_counters {
    int64_t submitted, admitted, solo, taken_out, completed, refused, slices, idle_solo;
} eg_server_counters;
eg_status eg_server_counters_get(eg_server *server, eg_server_counters *out);

/*
 * eg_server_set_option -- settings of a running server.
 *   EG_SRV_FAIL_RESERVATIONS (test hook, default 0): the next `value`
 *     reservations of pool room at admission fail as if the pool were full,
 *     so the refusal and retry path of admission can be exercised on the
 *     host without exhausting device memory.
 *   EG_SRV_IDLE_SOLO (default 1): a request that finds the server idle gets
 *     the single-game route's first attempt alone before it joins the pool;
 *     0 sends every request to the pool.
 * EG_ERR_INVALID for an unknown option or a value out of range.
 */
#define EG_SRV_FAIL_RESERVATIONS 1
#define EG_SRV_IDLE_SOLO 2
eg_status eg_server_set_option(eg_server *server, int32_t option, int64_t value);

/* eg_last_error -- message of the calling thread's last failure ("" if none). */
const char *eg_last_error(void);

/* eg_version -- library version string. */
const char *eg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EG_H */
