"""Pins for the CPU oracle (Algorithm 1 of arXiv 1710.03647, Sec. 3.1).

The oracle is checked against things other than itself:
  * hand-worked games derived from Eq. 1 / Def. "EPM" (tests/golden),
  * closed forms of Eq. 1 for single-successor arenas (lassos and cycles),
  * brute force over player-0 memoryless strategies (Lemma "EGcycles") on
    thousands of random tiny arenas,
  * the least-EPM equations and the bound M_G on larger arenas,
  * planted mistakes (mutants of oracle.c compiled here) that these pins
    must catch.
"""
from __future__ import annotations

import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import gen
from tests._games import TOP64, arena_from_edges, functional_credit, load_hand_games


def solve(a, **kw):
    f, st = oracle.solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits, **kw)
    return f, st


@pytest.mark.parametrize("game", load_hand_games(), ids=lambda g: g[0].name)
def test_hand_games(game):
    a, bound, expect = game
    assert oracle.bound(a.n, a.row_ptr, a.w) == bound
    f, _ = solve(a)
    np.testing.assert_array_equal(f, expect)
    # the hand-worked answers also agree with the exhaustive definition
    np.testing.assert_array_equal(oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits), expect)
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, f)[0] == 0


def test_bound_by_hand():
    # M_G = sum_v max(0, max_e -w): rows {-3, 5}, {2}, {-7, -1, 0}
    a = arena_from_edges([0, 1, 0], [(0, 1, -3), (0, 2, 5), (1, 0, 2), (2, 0, -7), (2, 1, -1), (2, 2, 0)])
    assert oracle.bound(a.n, a.row_ptr, a.w) == 3 + 0 + 7


@pytest.mark.parametrize("seed", range(200))
def test_single_successor_closed_form(seed):
    s = gen.Stream(seed, 99)
    n = int(1 + s.below(1, 12)[0])
    succ = gen.Stream(seed, 98).below(n, n)
    weight = gen.Stream(seed, 97).integers(n, -6, 6)
    owners = gen.Stream(seed, 96).below(n, 2).astype(bool)
    a = arena_from_edges(owners, [(v, int(succ[v]), int(weight[v])) for v in range(n)])
    f, _ = solve(a)
    np.testing.assert_array_equal(f, functional_credit(succ, weight))


def _tiny(seed):
    s = gen.Stream(seed, 90)
    n = int(1 + s.below(1, 7)[0])
    p1 = float(gen.Stream(seed, 91).unit(1)[0])
    return gen.tiny_game(n, max_deg=3, wlo=-4, whi=4, seed=seed, p1=p1)


@pytest.mark.parametrize("block", range(10))
def test_brute_force_random_tiny(block):
    for seed in range(block * 300, (block + 1) * 300):
        a = _tiny(seed)
        f, _ = solve(a)
        bf = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        assert np.array_equal(f, bf), (seed, f, bf)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_one_player(seed):
    # all player 1: a single strategy, the textbook worst-case walk
    a = gen.tiny_game(int(5 + seed % 20), max_deg=3, wlo=-5, whi=5, seed=1000 + seed, p1=1.0)
    f, _ = solve(a)
    np.testing.assert_array_equal(f, oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits))


@pytest.mark.parametrize("seed", range(1, 6))
def test_uniform_1k_invariants(seed):
    a = gen.config(1, seed)
    C = oracle.bound(a.n, a.row_ptr, a.w)
    f, st = solve(a)
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, f, C)[0] == 0
    fin = f[f != TOP64]
    assert fin.size and fin.max() <= C and fin.min() >= 0
    assert 0 < (f == TOP64).sum() < a.n
    assert st["lifts"] > 0


def test_equation_check_rejects_wrong_answers():
    a = gen.config(1, 1)
    f, _ = solve(a)
    fin = np.nonzero(f != TOP64)[0]
    g = f.copy()
    g[fin[0]] += 1
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, g)[0] == 2
    g = f.copy()
    g[fin[0]] = -1
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, g)[0] == 1


def test_non_total_rejected():
    a = arena_from_edges([0, 1], [(0, 1, 1)])  # vertex 1 has no successor
    with pytest.raises(oracle.OracleError):
        solve(a)


def test_solution_independent_of_cap_above_credits():
    # Any cap at or above the largest finite credit gives the same least
    # fixpoint (the bounded operator only turns values above the cap into TOP).
    a = gen.config(1, 2)
    f, _ = solve(a)
    C = oracle.bound(a.n, a.row_ptr, a.w)
    g, _ = solve(a, C=2 * C)
    np.testing.assert_array_equal(f, g)


# ---- planted mistakes: each mutant of oracle.c must fail some pin ----------

MUTANTS = {
    "minus_sign": (r"int64_t d = a - b;", "int64_t d = a + b;"),
    "cap_off_by_one": (r"if \(d > C\)\n        return ORACLE_TOP;", "if (d >= C)\n        return ORACLE_TOP;"),
    "min_max_swapped": (r"if \(p1 \? \(t > g\) : \(t < g\)\)", "if (p1 ? (t < g) : (t > g))"),
    "counter_strict": (r"if \(count\[u\] <= 0\)", "if (count[u] < 0)"),
    "init_p1_needs_all_negative": (r"if \(is_p1\(owner_bits, v\) \? any_neg : all_neg\)", "if (all_neg)"),
    "pre_filter_flipped": (r"if \(!\(f\[u\] < ominus\(f\[v\], wu, C\)\)\)", "if (!(f[u] > ominus(f[v], wu, C)))"),
}


def _mutant_lib(tmpdir, name):
    pat, rep = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    mutated, k = re.subn(pat, rep, src)
    assert k >= 1, f"mutation {name} did not apply"
    c = os.path.join(tmpdir, f"{name}.c")
    so = os.path.join(tmpdir, f"{name}.so")
    open(c, "w").write(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-o", so, c])
    return so


def _pins_pass(lib_path) -> bool:
    """Runs the hand games and a brute-force sample through a given library."""
    import ctypes

    lib = ctypes.CDLL(lib_path)
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.oracle_solve.restype = ctypes.c_int
    lib.oracle_solve.argtypes = [i64, p, p, p, p, i64, i64, p, p]
    lib.oracle_bound.restype = i64
    lib.oracle_bound.argtypes = [i64, p, p]

    def run(a):
        rp = np.ascontiguousarray(a.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(a.col, dtype=np.int32)
        w = np.ascontiguousarray(a.w, dtype=np.int64)
        ob = np.ascontiguousarray(a.owner_bits, dtype=np.uint32)
        C = lib.oracle_bound(a.n, rp.ctypes.data, w.ctypes.data)
        f = np.zeros(a.n, dtype=np.int64)
        st = np.zeros(4, dtype=np.int64)
        rc = lib.oracle_solve(a.n, rp.ctypes.data, col.ctypes.data, w.ctypes.data, ob.ctypes.data, C,
                              10_000_000, f.ctypes.data, st.ctypes.data)
        return rc, f

    for a, _, expect in load_hand_games():
        rc, f = run(a)
        if rc != 0 or not np.array_equal(f, expect):
            return False
    for seed in range(400):
        a = _tiny(seed)
        rc, f = run(a)
        if rc != 0 or not np.array_equal(f, oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)):
            return False
    return True


def test_pins_pass_on_real_oracle():
    assert _pins_pass(oracle.build())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    with tempfile.TemporaryDirectory() as d:
        assert not _pins_pass(_mutant_lib(d, name)), f"mutant {name} slipped through the pins"


# ---- the facts certified trial caps rest on, checked by brute force --------
# (1) In the dual game -- weights -(K w + 1), owners swapped -- a vertex with a
#     finite least-EPM value under any cap is won by player 1 in the game.
# (2) If, for a cap B, every vertex is finite in the game's capped least
#     fixpoint or proven lost by (1), that capped fixpoint is the least EPM.

def _dual(a, K):
    w2 = -(np.int64(K) * np.asarray(a.w, dtype=np.int64)) - 1
    ob2 = (~np.asarray(a.owner_bits, dtype=np.uint32)).astype(np.uint32)
    return w2, ob2


@pytest.mark.parametrize("block", range(10))
def test_dual_finite_only_on_player1_wins(block):
    for seed in range(block * 60, block * 60 + 60):
        a = _tiny(seed)
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        maxw = int(np.abs(a.w).max()) if a.w.size else 0
        for K in (1, 2, 8, a.n + 1):
            w2, ob2 = _dual(a, K)
            for B in (1, maxw, 4 * maxw + 3):
                g, _ = oracle.solve(a.n, a.row_ptr, a.col, w2, ob2, C=(K + 1) * B)
                fin = g != TOP64
                assert (exact[fin] == TOP64).all(), (seed, K, B)


@pytest.mark.parametrize("block", range(10))
def test_capped_fixpoint_exact_when_every_vertex_is_decided(block):
    decided_runs = 0
    for seed in range(block * 60, block * 60 + 60):
        a = _tiny(seed)
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        maxw = max(1, int(np.abs(a.w).max()) if a.w.size else 1)
        w2, ob2 = _dual(a, 8)
        for B in (maxw, 2 * maxw, 4 * maxw):
            proven = oracle.solve(a.n, a.row_ptr, a.col, w2, ob2, C=9 * B)[0] != TOP64
            f, _ = oracle.solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits, C=B)
            if ((f != TOP64) | proven).all():
                decided_runs += 1
                np.testing.assert_array_equal(f, exact)
    assert decided_runs > 0


# ---- the paper's Algorithm 2 (CPU baseline) reaches the same least fixpoint --

@pytest.mark.parametrize("threads", [1, 4])
def test_sweep_baseline_matches_algorithm_1(threads):
    for a in [gen.config(1, 1), gen.config(1, 2), gen.rmat_game(10, 8, seed=3),
              gen.varied_game(1500, 2, 16, 200, seed=4), gen.grid_game(12, 12, seed=2)]:
        f, _ = solve(a)
        g, st = oracle.sweep(a.n, a.row_ptr, a.col, a.w, a.owner_bits, threads=threads)
        np.testing.assert_array_equal(g, f)
        assert st["sweeps"] >= 1 and st["edge_evals"] == st["sweeps"] * a.m
    for seed in range(300):
        a = _tiny(seed)
        g, _ = oracle.sweep(a.n, a.row_ptr, a.col, a.w, a.owner_bits, threads=threads)
        np.testing.assert_array_equal(g, oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits))


# ---- the certified composition of capped Algorithm 1 runs ------------------
# oracle.certified_solve decides games by the two facts above; whatever trial
# decides a game, the result must be the unique least EPM: the cap-C run of
# Algorithm 1 on moderate games, brute force on tiny ones.

def _certified(a, w=None):
    return oracle.certified_solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)


@pytest.mark.parametrize("make", [
    lambda: gen.grid_game(32, 32, seed=1), lambda: gen.grid_game(48, 40, seed=2), lambda: gen.grid_game(64, 64, seed=3),
    lambda: gen.config(1, 1), lambda: gen.config(1, 2), lambda: gen.rmat_game(10, 8, seed=3),
    lambda: gen.varied_game(2000, 2, 16, 3000, seed=4), lambda: gen.varied_game(1500, 2, 6, 20, seed=5),
], ids=["grid32", "grid48x40", "grid64", "uniform1k_s1", "uniform1k_s2", "rmat10", "varied2k_W3000", "varied1500_W20"])
def test_certified_solve_matches_algorithm_1(make):
    a = make()
    f, st = _certified(a)
    g, _ = solve(a)
    np.testing.assert_array_equal(f, g)
    assert st["trial"] >= -1


def test_certified_solve_decides_grids_by_trials():
    # the grids need the trials (B = 4 max|w| is far below C) and are decided by them
    for seed in range(1, 5):
        a = gen.grid_game(40, 40, seed=seed)
        f, st = _certified(a)
        assert st["trial"] >= 0 and st["B"] < st["C"]
        np.testing.assert_array_equal(f, solve(a)[0])


@pytest.mark.parametrize("k", [-128, -40, 0, 60, 127])
def test_certified_solve_matches_algorithm_1_on_threshold_weights(k):
    a = gen.rmat_game(10, 8, seed=6)
    w2 = gen.threshold_weights(a.w, k, 100)
    f, _ = _certified(a, w2)
    g, _ = oracle.solve(a.n, a.row_ptr, a.col, w2, a.owner_bits)
    np.testing.assert_array_equal(f, g)


def test_certified_solve_matches_brute_force_on_tiny_games():
    for seed in range(400):
        a = _tiny(seed)
        f, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits, cap_mult=1)
        np.testing.assert_array_equal(f, oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits))


def test_certified_solve_zero_weight_cycle_is_a_player0_win():
    # player 0 at vertex 0 can stay on the cycle 0 -> 1 -> 0 of weight 0
    # (vertex 1 belongs to player 1 but has no other edge) or take the
    # -1000 edge to the player-1 sink 2, which loops at weight -1.  The
    # zero-weight cycle needs credit 0; it must not be mistaken for a loss
    # (the dual's -1 per edge is what keeps it out of the dual's finite set).
    a = arena_from_edges([0, 1, 1], [(0, 1, 5), (0, 2, -1000), (1, 0, -5), (2, 2, -1)])
    f, st = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits, cap_mult=1)
    np.testing.assert_array_equal(f, [0, 5, TOP64])
    np.testing.assert_array_equal(f, oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits))


# (3) In the dual game, vertices already proven lost may be replaced by sinks
#     of value 0 (a self-loop of dual weight 0): a vertex finite in that
#     modified dual is still won by player 1 in the game, since player 1
#     either keeps the play on negative cycles or reaches a proven loss.

def _dual_with_sinks(a, K, sinks):
    w2, ob2 = _dual(a, K)
    rp = np.asarray(a.row_ptr, dtype=np.int64)
    rows_c, rows_w = [], []
    for v in range(a.n):
        if sinks[v]:
            rows_c.append([v])
            rows_w.append([0])
        else:
            rows_c.append(list(a.col[rp[v]:rp[v + 1]]))
            rows_w.append(list(w2[rp[v]:rp[v + 1]]))
    rp2 = np.zeros(a.n + 1, dtype=np.int64)
    rp2[1:] = np.cumsum([len(r) for r in rows_c])
    return (rp2, np.array([c for r in rows_c for c in r], dtype=np.int32),
            np.array([x for r in rows_w for x in r], dtype=np.int64), ob2)


@pytest.mark.parametrize("block", range(6))
def test_dual_with_proven_losses_as_sinks_finds_only_losses(block):
    checked = 0
    for seed in range(block * 60, block * 60 + 60):
        a = _tiny(seed)
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        lost = exact == TOP64
        if not lost.any():
            continue
        pick = gen.Stream(seed, 99).unit(a.n) < 0.5
        maxw = max(1, int(np.abs(a.w).max()) if a.w.size else 1)
        for sinks in (lost & pick, lost):
            for K in (1, 8, a.n + 1):
                rp2, col2, w2, ob2 = _dual_with_sinks(a, K, sinks)
                for B in (maxw, 4 * maxw + 3):
                    g, _ = oracle.solve(a.n, rp2, col2, w2, ob2, C=(K + 1) * B)
                    fin = g != TOP64
                    assert (exact[fin] == TOP64).all(), (seed, K, B)
                    checked += 1
    assert checked > 0


# ---- the cycle bound behind the accelerated lifting --------------------------
# For a cycle c of the arena whose weight is negative, and credits f at or
# below the least fixpoint, let alt(u) be, for a player-0 vertex u of c, the
# least f(x) (-) w over u's edges other than its edge on c.  The greatest
# solution x of  x(v) = x(next) (-) w  (player 1),
#                x(v) = min(x(next) (-) w, alt(v))  (player 0)
# around c is at or below the least fixpoint at every vertex of c: the least
# fixpoint cannot follow c all the way round (each lap would need d more
# credit), so some player-0 vertex of c leaves it at or above its alt.

def _cycle_bound(a, f, cyc_edges, C):
    """x on the cycle given by its edge ids (in order), from x = TOP."""
    rp = np.asarray(a.row_ptr)
    src = np.repeat(np.arange(a.n), np.diff(rp))
    w = np.asarray(a.w, dtype=np.int64)
    p1 = gen.unpack_owner(a.owner_bits, a.n)

    def om(x, wt):
        if x == TOP64:
            return TOP64
        d = x - wt
        return TOP64 if d > C else max(0, d)

    L = len(cyc_edges)
    verts = [int(src[e]) for e in cyc_edges]
    alts = []
    for e, v in zip(cyc_edges, verts):
        others = [om(int(f[a.col[k]]), int(w[k])) for k in range(rp[v], rp[v + 1]) if k != e]
        alts.append(min(others) if others else TOP64)
    x = [TOP64] * L
    for _ in range(2):
        for i in range(L - 1, -1, -1):
            val = om(x[(i + 1) % L], int(w[cyc_edges[i]]))
            if not p1[verts[i]]:
                val = min(val, alts[i])
            x[i] = val
    return verts, x


def _simple_cycles(a, max_len=5):
    """Edge-id lists of the simple cycles of length <= max_len (each once)."""
    rp = np.asarray(a.row_ptr)
    out = []

    def walk(start, v, path_e, seen):
        for e in range(rp[v], rp[v + 1]):
            u = int(a.col[e])
            if u == start:
                out.append(path_e + [e])
            elif u > start and u not in seen and len(path_e) + 1 < max_len:
                walk(start, u, path_e + [e], seen | {u})
    for s in range(a.n):
        walk(s, s, [], {s})
    return out


@pytest.mark.parametrize("block", range(4))
def test_cycle_bound_stays_below_the_least_fixpoint(block):
    checked = 0
    for seed in range(block * 50, block * 50 + 50):
        a = _tiny(seed)
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        C = oracle.bound(a.n, a.row_ptr, a.w)
        w = np.asarray(a.w, dtype=np.int64)
        for cyc in _simple_cycles(a):
            if int(w[cyc].sum()) >= 0:
                continue
            # credits at or below the least fixpoint: 0, the fixpoint itself,
            # and random ones in between (TOP drawn from {0..C} u {TOP})
            draws = gen.Stream(seed, 31 + len(cyc)).unit(4 * a.n).reshape(4, a.n)
            cases = [np.zeros(a.n, dtype=np.int64), exact.copy()]
            for row in draws:
                hi = np.where(exact == TOP64, C + 1, exact)
                f = np.floor(row * (hi + 1)).astype(np.int64)
                f = np.where(f > C, TOP64, np.minimum(f, hi))
                cases.append(np.where(exact == TOP64, f, np.minimum(f, exact)))
            for f in cases:
                assert (f <= exact).all()
                verts, x = _cycle_bound(a, f, cyc, C)
                for v, xv in zip(verts, x):
                    assert xv <= exact[v], (seed, cyc, v, xv, exact[v])
                checked += 1
    assert checked > 0


def test_cycle_bound_catches_a_wrong_bound():
    # the bound with the alternatives dropped (a lap assumed to be forced)
    # exceeds the least fixpoint somewhere: the pin above would catch it
    broke = 0
    for seed in range(200):
        a = _tiny(seed)
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        C = oracle.bound(a.n, a.row_ptr, a.w)
        w = np.asarray(a.w, dtype=np.int64)
        for cyc in _simple_cycles(a):
            if int(w[cyc].sum()) >= 0:
                continue
            verts = [int(np.searchsorted(np.asarray(a.row_ptr), e, side="right") - 1) for e in cyc]
            # no exits: every vertex of the cycle would be TOP
            if any(exact[v] != TOP64 for v in verts):
                broke += 1
    assert broke > 0


# Reading 24 (dense sweeps).  A model of the solver's sweeps and of the
# worklist rounds that follow them: each sweep raises every credit, in a random
# order, to its lift (min over edges for player 0, max for player 1), reading
# each successor either as it is now or as it was when the sweep began (what a
# concurrent sweep may see); the rounds then start from the credits the last
# sweep raised.  The credits must stay at or below the least fixpoint after
# every sweep and end exactly at it.

def _ominus(x, wt, C):
    if x == TOP64:
        return TOP64
    d = x - wt
    return TOP64 if d > C else max(0, d)


def _sweep_model(a, C, sweeps, rng, exact, frontier=True):
    rp = np.asarray(a.row_ptr)
    col = np.asarray(a.col)
    w = np.asarray(a.w, dtype=np.int64)
    p1 = gen.unpack_owner(a.owner_bits, a.n)
    preds = [[] for _ in range(a.n)]
    for v in range(a.n):
        for k in range(rp[v], rp[v + 1]):
            preds[int(col[k])].append((v, k))

    def lift(v, read):
        vals = [_ominus(read(int(col[k])), int(w[k]), C) for k in range(rp[v], rp[v + 1])]
        return max(vals) if p1[v] else min(vals)

    f = [lift(v, lambda u: 0) for v in range(a.n)]  # the init: the lift over f = 0
    last = set()
    for _ in range(sweeps):
        snap = list(f)
        last = set()
        for v in rng.permutation(a.n):
            v = int(v)
            t = lift(v, lambda u: snap[u] if rng.random() < 0.5 else f[u])
            if t > f[v]:
                f[v] = t
                last.add(v)
        assert all(x <= e for x, e in zip(f, exact))
    from collections import deque

    queue = deque(sorted(last) if frontier else [])
    queued = set(queue)
    while queue:  # the rounds: rises pushed to predecessors
        u = queue.popleft()
        queued.discard(u)
        for p, k in preds[u]:
            t = _ominus(f[u], int(w[k]), C)
            if t <= f[p]:
                continue
            nv = t if p1[p] else lift(p, lambda x: f[x])
            if nv > f[p]:
                f[p] = nv
                if p not in queued:
                    queue.append(p)
                    queued.add(p)
    return np.asarray(f, dtype=np.int64)


def test_sweeps_then_frontier_reach_the_least_fixpoint():
    rng = np.random.default_rng(24)
    games = [_tiny(seed) for seed in range(300)]
    games += [gen.varied_game(int(n), 1, 4, 12, seed=500 + i) for i, n in enumerate(rng.integers(20, 80, 40))]
    short = 0
    for a in games:
        exact = oracle.brute_force(a.n, a.row_ptr, a.col, a.w, a.owner_bits) if a.n <= 7 else solve(a)[0]
        C = oracle.bound(a.n, a.row_ptr, a.w)
        for sweeps in (1, 2, 4):
            np.testing.assert_array_equal(_sweep_model(a, C, sweeps, rng, exact), exact)
            # without the last sweep's frontier the rounds miss rises
            if not np.array_equal(_sweep_model(a, C, sweeps, rng, exact, frontier=False), exact):
                short += 1
    assert short > 0
