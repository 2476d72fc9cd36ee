/*
 * Algorithm 2 of arXiv 1710.03647 (Sec. 4, "An OpenMP implementation"): the
 * paper's multi-core baseline for the initial credit problem.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: a CPU baseline that the benchmark
 * times beside the GPU solver (the paper's CPU EG8 column is this algorithm
 * on 8 threads).  Nothing on the product path may link, load or call it, and
 * it shares no code with the CUDA sources or with oracle.c.
 *
 * Starting from f = 0, every sweep applies the lifting operator of Def.
 * "Lifting Operator" to all vertices in parallel, in place, until a sweep
 * changes nothing or max_sweeps sweeps ran (the paper stops at |E| * M_G).
 * Lifts never decrease f, so lifting in place and in parallel is sound (the
 * paper's argument for running the loop in parallel).  In one sweep each
 * vertex is written by the one thread that lifts it; reads of other vertices
 * are relaxed atomic loads, so a thread may see a neighbour's value of this
 * sweep or of the last one -- either is at most the least fixpoint.
 *
 * (-) is bounded by the codomain {0..C} u {TOP} of Sec. 3.1; TOP is
 * INT64_MAX.
 */
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SWEEP_TOP INT64_MAX

static int64_t bounded_minus(int64_t a, int64_t b, int64_t C)
{
    if (a == SWEEP_TOP)
        return SWEEP_TOP;
    int64_t d = a - b;
    if (d > C)
        return SWEEP_TOP;
    return d < 0 ? 0 : d;
}

/*
 * Returns 0 at the fixpoint, 1 if a vertex has no successor, 2 if
 * max_sweeps > 0 sweeps did not reach it.  stats (may be NULL), 3 entries:
 * sweeps, edge evaluations, threads used.  threads <= 0: the OpenMP default.
 */
int oracle_sweep(int64_t n, const int64_t *row_ptr, const int32_t *col, const int64_t *w,
                 const uint32_t *owner_bits, int64_t C, int64_t max_sweeps, int threads,
                 int64_t *f, int64_t *stats)
{
    for (int64_t v = 0; v < n; ++v) {
        if (row_ptr[v + 1] == row_ptr[v])
            return 1;
        f[v] = 0;
    }
    int used = 1;
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#endif
    int64_t sweeps = 0, evals = 0;
    int more = 1;
    while (more && (max_sweeps <= 0 || sweeps < max_sweeps)) {
        more = 0;
        ++sweeps;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : more)
        for (int64_t v = 0; v < n; ++v) {
            const int p1 = (int)((owner_bits[v >> 5] >> (v & 31)) & 1u);
            int64_t g = p1 ? 0 : SWEEP_TOP;
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                const int64_t t = bounded_minus(__atomic_load_n(&f[col[e]], __ATOMIC_RELAXED), w[e], C);
                if (p1 ? (t > g) : (t < g))
                    g = t;
            }
            if (g > __atomic_load_n(&f[v], __ATOMIC_RELAXED)) {
                __atomic_store_n(&f[v], g, __ATOMIC_RELAXED);
                more = 1;
            }
        }
        evals += row_ptr[n];
    }
    if (stats) {
        stats[0] = sweeps;
        stats[1] = evals;
        stats[2] = used;
    }
    return more ? 2 : 0;
}
