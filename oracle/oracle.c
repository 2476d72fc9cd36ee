/*
 * CPU oracle for the initial credit problem of energy games.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can check the CUDA solver against a plain,
 * slow, single-threaded restatement of the paper.  It shares no code,
 * header or table with the CUDA sources.
 *
 * Paper: A. Formisano, R. Gentilini, F. Vella, "Accelerating Energy Games
 * Solvers on Modern Architectures" (arXiv 1710.03647).
 *
 *   oracle_bound        the bound M_G of Sec. 3.1 (sum over vertices of the
 *                       largest negated out-weight, floored at 0)
 *   oracle_solve        Algorithm 1 (Sec. 3.1): FIFO worklist with the
 *                       player-0 counters, lifting operator of Def. "Lifting
 *                       Operator", bounded (-) of Sec. 3.1 with codomain C_G
 *   oracle_brute_force  independent check via Lemma "EGcycles" (Sec. 3):
 *                       enumerate player-0 memoryless strategies, then a
 *                       Bellman-Ford worst case in the one-player graph
 *   oracle_check        the least-EPM equations of Def. "EPM" / "Lifting
 *                       Operator" and the range {0..C} u {TOP}
 *
 * Credits are int64 with TOP = INT64_MAX (the largest value, so the order of
 * Sec. 3.1 is the numeric order).  Weights are int64 so that shifted
 * threshold weights fit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TOP INT64_MAX

static int is_p1(const uint32_t *owner_bits, int64_t v)
{
    return (int)((owner_bits[v >> 5] >> (v & 31)) & 1u);
}

/* a (-) b of Sec. 3.1, bounded by the codomain C_G = {0..C} u {TOP}:
 * TOP stays TOP, a value above C becomes TOP, a negative one becomes 0. */
static int64_t ominus(int64_t a, int64_t b, int64_t C)
{
    if (a == ORACLE_TOP)
        return ORACLE_TOP;
    int64_t d = a - b;
    if (d > C)
        return ORACLE_TOP;
    return d < 0 ? 0 : d;
}

/* M_G = sum over v of max({0} u {-w(v,v') : (v,v') in E}). */
int64_t oracle_bound(int64_t n, const int64_t *row_ptr, const int64_t *w)
{
    int64_t total = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t worst = 0;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (-w[e] > worst)
                worst = -w[e];
        total += worst;
    }
    return total;
}

/* delta(f, v)(v) of Def. "Lifting Operator": min over successors for a
 * player-0 vertex, max for a player-1 vertex, of f(v') (-) w(v, v'). */
static int64_t lift_value(int64_t v, int p1, const int64_t *row_ptr, const int32_t *col,
                          const int64_t *w, const int64_t *f, int64_t C)
{
    int64_t g = p1 ? 0 : ORACLE_TOP;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        int64_t t = ominus(f[col[e]], w[e], C);
        if (p1 ? (t > g) : (t < g))
            g = t;
    }
    return g;
}

/* |{v' in post(v) : f(v) >= f(v') (-) w(v, v')}|, counted over edges. */
static int64_t witnesses(int64_t v, const int64_t *row_ptr, const int32_t *col,
                         const int64_t *w, const int64_t *f, int64_t C)
{
    int64_t k = 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
        if (f[v] >= ominus(f[col[e]], w[e], C))
            ++k;
    return k;
}

/*
 * Algorithm 1.  Returns 0 on success, 1 if a vertex has no successor
 * (the arena is not total, Sec. 2), 2 if max_lifts > 0 lifts did not reach
 * the fixpoint, 3 on allocation failure.
 *
 * stats (may be NULL), 4 entries: lifts, edge evaluations inside lifts,
 * predecessor edges scanned, counter recount evaluations.
 */
int oracle_solve(int64_t n, const int64_t *row_ptr, const int32_t *col, const int64_t *w,
                 const uint32_t *owner_bits, int64_t C, int64_t max_lifts,
                 int64_t *f, int64_t *stats)
{
    for (int64_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] <= row_ptr[v])
            return 1;
    int64_t m = row_ptr[n];

    /* pre(v) as its own reverse adjacency: incoming edge list per vertex,
     * each entry the source v' and the weight w(v', v). */
    int64_t *pre_ptr = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *pre_src = malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    int64_t *pre_w = malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    int64_t *count = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *queue = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    char *in_l = calloc((size_t)(n ? n : 1), 1);
    int64_t *fill = malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!pre_ptr || !pre_src || !pre_w || !count || !queue || !in_l || !fill) {
        free(pre_ptr); free(pre_src); free(pre_w); free(count); free(queue); free(in_l); free(fill);
        return 3;
    }
    for (int64_t e = 0; e < m; ++e)
        pre_ptr[col[e] + 1]++;
    for (int64_t v = 0; v < n; ++v)
        pre_ptr[v + 1] += pre_ptr[v];
    memcpy(fill, pre_ptr, (size_t)n * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int64_t slot = fill[col[e]]++;
            pre_src[slot] = v;
            pre_w[slot] = w[e];
        }

    int64_t head = 0, size = 0; /* FIFO ring of capacity n with set semantics */
#define PUSH(x) do { if (!in_l[(x)]) { in_l[(x)] = 1; queue[(head + size) % n] = (x); ++size; } } while (0)

    /* the initial set L of Algorithm 1 */
    for (int64_t v = 0; v < n; ++v) {
        int any_neg = 0, all_neg = 1;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            if (w[e] < 0)
                any_neg = 1;
            else
                all_neg = 0;
        }
        if (is_p1(owner_bits, v) ? any_neg : all_neg)
            PUSH(v);
    }
    /* f = 0 and the player-0 counters */
    for (int64_t v = 0; v < n; ++v)
        f[v] = 0;
    int64_t recount_evals = 0;
    for (int64_t v = 0; v < n; ++v) {
        count[v] = 0;
        if (!is_p1(owner_bits, v) && !in_l[v]) {
            count[v] = witnesses(v, row_ptr, col, w, f, C);
            recount_evals += row_ptr[v + 1] - row_ptr[v];
        }
    }

    int64_t lifts = 0, lift_evals = 0, pre_scans = 0;
    int status = 0;
    /* the worklist loop: lift, recount, predecessor filter */
    while (size > 0) {
        if (max_lifts > 0 && lifts >= max_lifts) {
            status = 2;
            break;
        }
        int64_t v = queue[head];
        head = (head + 1) % n;
        --size;
        in_l[v] = 0;
        int p1 = is_p1(owner_bits, v);
        int64_t old = f[v];
        f[v] = lift_value(v, p1, row_ptr, col, w, f, C);
        ++lifts;
        lift_evals += row_ptr[v + 1] - row_ptr[v];
        if (!p1) {
            count[v] = witnesses(v, row_ptr, col, w, f, C);
            recount_evals += row_ptr[v + 1] - row_ptr[v];
        }
        for (int64_t s = pre_ptr[v]; s < pre_ptr[v + 1]; ++s) {
            int64_t u = pre_src[s];
            int64_t wu = pre_w[s];
            ++pre_scans;
            if (!(f[u] < ominus(f[v], wu, C)))
                continue;
            if (!is_p1(owner_bits, u)) {
                if (f[u] >= ominus(old, wu, C))
                    count[u] -= 1;
                if (count[u] <= 0)
                    PUSH(u);
            } else {
                PUSH(u);
            }
        }
    }
#undef PUSH
    if (stats) {
        stats[0] = lifts;
        stats[1] = lift_evals;
        stats[2] = pre_scans;
        stats[3] = recount_evals;
    }
    free(pre_ptr); free(pre_src); free(pre_w); free(count); free(queue); free(in_l); free(fill);
    return status;
}

/*
 * Exhaustive check for tiny arenas (Lemma "EGcycles", Sec. 3).
 *
 * For every player-0 memoryless strategy pi0 (one successor edge per
 * player-0 vertex) the graph G(pi0) keeps that edge for player-0 vertices
 * and every edge for player-1 vertices.  In G(pi0), from a source v:
 *   - if a negative cycle is reachable from v, pi0 does not win from v;
 *   - otherwise every play consistent with pi0 keeps the energy level
 *     c + (prefix sum) >= 0 iff c >= -(shortest walk from v), and the
 *     shortest walk equals the Bellman-Ford shortest-path distance, so the
 *     credit under pi0 is max(0, -min_u dist(v, u)).
 * The minimum initial credit is the minimum over pi0 (memoryless
 * strategies suffice for player 0 in energy games); TOP when no pi0 wins.
 *
 * Returns 0, 1 if a vertex has no successor, 2 if the number of strategies
 * exceeds max_strategies, 3 on allocation failure.
 */
int oracle_brute_force(int64_t n, const int64_t *row_ptr, const int32_t *col, const int64_t *w,
                       const uint32_t *owner_bits, int64_t max_strategies, int64_t *credit)
{
    int64_t m = row_ptr[n];
    int64_t strategies = 1;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d <= 0)
            return 1;
        if (!is_p1(owner_bits, v)) {
            if (strategies > max_strategies / d)
                return 2;
            strategies *= d;
        }
    }
    int64_t *choice = calloc((size_t)n + 1, sizeof(int64_t));
    char *keep = malloc((size_t)(m ? m : 1));
    int64_t *dist = malloc((size_t)n * sizeof(int64_t));
    char *seen = malloc((size_t)n);
    if (!choice || !keep || !dist || !seen) {
        free(choice); free(keep); free(dist); free(seen);
        return 3;
    }
    for (int64_t v = 0; v < n; ++v)
        credit[v] = ORACLE_TOP;
    const int64_t INF = INT64_MAX;

    for (int64_t s = 0; s < strategies; ++s) {
        /* decode strategy index s as mixed-radix digits over player-0 vertices */
        int64_t rest = s;
        for (int64_t v = 0; v < n; ++v) {
            int64_t d = row_ptr[v + 1] - row_ptr[v];
            if (is_p1(owner_bits, v)) {
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                    keep[e] = 1;
            } else {
                choice[v] = rest % d;
                rest /= d;
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                    keep[e] = (e - row_ptr[v]) == choice[v];
            }
        }
        for (int64_t src = 0; src < n; ++src) {
            for (int64_t u = 0; u < n; ++u) {
                dist[u] = INF;
                seen[u] = 0;
            }
            dist[src] = 0;
            /* n - 1 rounds of relaxation over every kept edge */
            for (int64_t it = 0; it + 1 < n; ++it) {
                int changed = 0;
                for (int64_t u = 0; u < n; ++u) {
                    if (dist[u] == INF)
                        continue;
                    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                        if (keep[e] && dist[u] + w[e] < dist[col[e]]) {
                            dist[col[e]] = dist[u] + w[e];
                            changed = 1;
                        }
                }
                if (!changed)
                    break;
            }
            /* one more round: any improvement means a reachable negative cycle */
            int neg_cycle = 0;
            for (int64_t u = 0; u < n && !neg_cycle; ++u) {
                if (dist[u] == INF)
                    continue;
                for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                    if (keep[e] && dist[u] + w[e] < dist[col[e]]) {
                        neg_cycle = 1;
                        break;
                    }
            }
            if (neg_cycle)
                continue;
            int64_t lowest = 0;
            for (int64_t u = 0; u < n; ++u)
                if (dist[u] != INF && dist[u] < lowest)
                    lowest = dist[u];
            if (-lowest < credit[src])
                credit[src] = -lowest;
        }
    }
    free(choice); free(keep); free(dist); free(seen);
    return 0;
}

/*
 * Checks a claimed least EPM f: every value lies in {0..C} u {TOP} and every
 * vertex satisfies the lifting equation f(v) = delta(f, v)(v) (which implies
 * the EPM conditions of Def. "EPM").  Returns 0 if all hold, 1 for a value
 * out of range, 2 for a failed equation; *bad receives the first bad vertex.
 */
int oracle_check(int64_t n, const int64_t *row_ptr, const int32_t *col, const int64_t *w,
                 const uint32_t *owner_bits, int64_t C, const int64_t *f, int64_t *bad)
{
    for (int64_t v = 0; v < n; ++v) {
        if (f[v] != ORACLE_TOP && (f[v] < 0 || f[v] > C)) {
            *bad = v;
            return 1;
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        if (lift_value(v, is_p1(owner_bits, v), row_ptr, col, w, f, C) != f[v]) {
            *bad = v;
            return 2;
        }
    }
    *bad = -1;
    return 0;
}
