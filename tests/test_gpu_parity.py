"""GPU parity: the CUDA solver (through the C ABI) against the CPU oracle.

Credits are integers, so every comparison is exact (tolerance 0), element by
element, for both credit widths.  The oracle itself is pinned by
tests/test_oracle_pins.py (brute force, closed forms, hand-worked games).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen
from tests._games import GOLDEN, TOP64, arena_from_edges, load_hand_games

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def ref(a, w=None):
    w = a.w if w is None else w
    f, _ = oracle.solve(a.n, a.row_ptr, a.col, w, a.owner_bits)
    return f


def gpu(a, bits=0, scale=1, shift=0, max_rounds=0, rev=None, **opts):
    with eg.Arena(a, with_reverse=rev) as ar:
        if opts:
            ar.tune(**opts)
        out, st = ar.solve(credit_bits=bits, w_scale=scale, w_shift=shift, max_rounds=max_rounds)
    return out, st


def as64(f, bits):
    f = np.asarray(f)
    if bits == 32:
        return np.where(f == eg.EG_TOP32, TOP64, f.astype(np.int64))
    return f


@pytest.mark.parametrize("bits", [0, 32, 64])
@pytest.mark.parametrize("game", load_hand_games(), ids=lambda g: g[0].name)
def test_hand_games(game, bits):
    a, bound, expect = game
    out, st = gpu(a, bits)
    np.testing.assert_array_equal(as64(out, bits), expect)
    assert st.C == bound
    assert st.credit_bits == (bits or 32)


def test_tiny_random_games():
    for seed in range(300):
        s = gen.Stream(seed, 90)
        n = int(1 + s.below(1, 7)[0])
        a = gen.tiny_game(n, max_deg=3, wlo=-4, whi=4, seed=seed, p1=float(gen.Stream(seed, 91).unit(1)[0]))
        out, _ = gpu(a)
        assert np.array_equal(out, ref(a)), seed


@pytest.mark.parametrize("bits", [0, 32, 64])
@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_uniform_1k(seed, bits):
    a = gen.config(1, seed)
    out, st = gpu(a, bits)
    np.testing.assert_array_equal(as64(out, bits), ref(a))
    assert st.rounds > 0 and st.relaxations > 0


@pytest.mark.parametrize("scale", [10, 12, 14])
def test_rmat_scaled(scale):
    a = gen.rmat_game(scale, 8, seed=3)
    out, _ = gpu(a)
    np.testing.assert_array_equal(out, ref(a))


@pytest.mark.parametrize("rows,cols", [(32, 32), (48, 80), (64, 64)])
def test_grid_scaled(rows, cols):
    a = gen.grid_game(rows, cols, seed=2)
    out, _ = gpu(a, 64)
    np.testing.assert_array_equal(out, ref(a))


@pytest.mark.parametrize("n,dlo,dhi,W", [(3000, 2, 16, 10), (5000, 2, 16, 10000), (777, 2, 16, 300)])
def test_varied_games(n, dlo, dhi, W):
    a = gen.varied_game(n, dlo, dhi, W, seed=n)
    out, _ = gpu(a)
    np.testing.assert_array_equal(out, ref(a))


@pytest.mark.parametrize("k", [-128, -7, 0, 1, 5, 127])
def test_threshold_queries(k):
    # w' = 256 w - k W, applied on the fly by the solver
    a = gen.rmat_game(11, 8, seed=5)
    W = 100
    wq = gen.threshold_weights(a.w, k, W)
    out, st = gpu(a, 0, scale=256, shift=k * W)
    np.testing.assert_array_equal(out, ref(a, wq))
    assert st.C == oracle.bound(a.n, a.row_ptr, wq)


def test_all_player0_and_all_player1():
    base = gen.uniform_game(2000, 4, -10, 10, seed=11)
    for p1 in (False, True):
        a = gen.Arena(base.n, base.row_ptr, base.col, base.w, gen.pack_owner(np.full(base.n, p1)))
        out, _ = gpu(a)
        np.testing.assert_array_equal(out, ref(a))


def test_single_vertex_loops():
    for owner in (0, 1):
        for wt in (-3, -1, 0, 2):
            a = arena_from_edges([owner], [(0, 0, wt)])
            out, _ = gpu(a)
            assert out[0] == (TOP64 if wt < 0 else 0)


def test_star_hub_split_across_warps():
    # vertex 0: 150k out-edges and 150k in-edges, so both phases cut its
    # scan across many warps and merge partial minima.  Leaf edges are
    # nonnegative, which keeps the bound C (and so the number of rounds) small.
    n = 150001
    s = gen.Stream(7, 1)
    edges = [(0, v, int(x)) for v, x in zip(range(1, n), s.integers(n - 1, -50, 50))]
    edges += [(v, 0, int(x)) for v, x in zip(range(1, n), gen.Stream(7, 2).integers(n - 1, 0, 50))]
    edges += [(v, v, int(x)) for v, x in zip(range(1, n), gen.Stream(7, 3).integers(n - 1, 0, 5))]
    for p1_center in (False, True):
        owners = (gen.Stream(7, 4).unit(n) < 0.5)
        owners[0] = p1_center
        a = arena_from_edges(owners, edges)
        out, _ = gpu(a)
        np.testing.assert_array_equal(out, ref(a))


def test_long_chain_many_rounds():
    # v -> v+1 with weight -1, last vertex a 0 self-loop: credit n-1-v
    n = 20000
    edges = [(v, v + 1, -1) for v in range(n - 1)] + [(n - 1, n - 1, 0)]
    a = arena_from_edges(np.zeros(n, dtype=bool), edges)
    out, st = gpu(a)
    np.testing.assert_array_equal(out, np.arange(n - 1, -1, -1, dtype=np.int64))
    assert st.rounds >= 1


def test_duplicate_edges_and_self_loops():
    a = gen.tiny_game(300, max_deg=6, wlo=-6, whi=6, seed=77, self_loops=True)
    out, _ = gpu(a)
    np.testing.assert_array_equal(out, ref(a))


def _reverse_csr(a):
    src = np.repeat(np.arange(a.n, dtype=np.int64), np.diff(a.row_ptr))
    order = np.argsort(a.col, kind="stable")
    rrow = np.zeros(a.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(a.col, minlength=a.n), out=rrow[1:])
    return rrow, src[order].astype(np.int32), a.w[order].astype(np.int32)


def test_caller_reverse_csr():
    a = gen.config(1, 3)
    rev = _reverse_csr(a)
    out, _ = gpu(a, rev=rev)
    np.testing.assert_array_equal(out, ref(a))
    bad = (rev[0], rev[1], rev[2].copy())
    bad[2][5] += 1
    with pytest.raises(eg.EGError) as ei:
        gpu(a, rev=bad)
    assert ei.value.status == eg.EG_ERR_INVALID


def test_malformed_inputs_rejected():
    a = arena_from_edges([0, 1, 0], [(0, 1, 1), (1, 2, -1), (2, 0, 3)])
    # vertex without successor
    rp = np.array([0, 1, 1, 2], dtype=np.int64)
    with pytest.raises(eg.EGError) as ei:
        eg.eg_create(3, 2, rp, np.array([1, 0], np.int32), np.array([1, 1], np.int32), owner_bits=a.owner_bits)
    assert ei.value.status == eg.EG_ERR_NOT_TOTAL
    # successor out of range
    with pytest.raises(eg.EGError) as ei:
        eg.eg_create(3, 3, a.row_ptr, np.array([1, 2, 3], np.int32), a.w, owner_bits=a.owner_bits)
    assert ei.value.status == eg.EG_ERR_INVALID
    # decreasing offsets
    with pytest.raises(eg.EGError) as ei:
        eg.eg_create(3, 3, np.array([0, 2, 1, 3], np.int64), a.col, a.w, owner_bits=a.owner_bits)
    assert ei.value.status == eg.EG_ERR_INVALID


def test_int32_overflow_reported():
    big = 2 ** 30
    a = arena_from_edges([1, 1, 0], [(0, 1, -big), (1, 2, -big), (2, 2, 0)])
    with pytest.raises(eg.EGError) as ei:
        gpu(a, 32)
    assert ei.value.status == eg.EG_ERR_OVERFLOW
    out, st = gpu(a, 0)
    assert st.credit_bits == 64
    np.testing.assert_array_equal(out, ref(a))


def test_round_budget_then_full_solve():
    a = gen.config(1, 4)
    with eg.Arena(a) as ar:
        ar.tune(warm_start=0, local_windows=0)  # one hop per round: needs many rounds
        out = np.empty(a.n, dtype=np.int64)
        rc, st = eg.eg_solve_credit(ar.handle, 0, 1, 0, out, max_rounds=3, raise_on_error=False)
        assert rc == eg.EG_ERR_BUDGET and st.rounds == 3
        full, st2 = ar.solve(0)
    np.testing.assert_array_equal(full, ref(a))
    # every partial value is below the fixpoint
    assert np.all(out <= full)


def test_repeat_solves_identical():
    a = gen.rmat_game(12, 8, seed=9)
    with eg.Arena(a) as ar:
        r1, _ = ar.solve(0)
        r2, _ = ar.solve(32)
        r3, _ = ar.solve(64)
    np.testing.assert_array_equal(r1, r3)
    np.testing.assert_array_equal(as64(r2, 32), r1)


def test_device_pointers_in_and_out():
    torch = pytest.importorskip("torch")
    a = gen.config(1, 5)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
         dict(rp=a.row_ptr, col=a.col, w=a.w, own=a.owner_bits.view(np.int32)).items()}
    h = eg.eg_create(a.n, a.m, t["rp"], t["col"], t["w"], owner_bits=t["own"], flags=eg.EG_INPUT_DEVICE)
    try:
        out = torch.empty(a.n, dtype=torch.int64, device=dev)
        stream = torch.cuda.Stream()
        eg.eg_solve_credit(h, 64, 1, 0, out, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref(a))
    finally:
        eg.eg_destroy(h)


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle result {name}.json")
    return json.load(open(path))


@pytest.mark.parametrize("name,make", [("rmat18_s1", lambda: gen.rmat_game(18, 8, seed=1)),
                                       ("rmat20_s1", lambda: gen.config(2, seed=1))])
def test_rmat_full_size_against_stored_oracle(name, make):
    g = _golden(name)
    a = make()
    out, st = gpu(a, 0)
    assert hashlib.sha256(out.astype(np.int64).tobytes()).hexdigest() == g["sha256"]
    assert st.C == g["C"]
    # and the least-EPM equations hold at every vertex (checked by the oracle)
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, out)[0] == 0


SCHEDULES = [dict(warm_start=0, local_windows=0), dict(warm_start=0, local_windows=64),
             dict(warm_start=1, local_windows=0), dict(warm_start=1, local_windows=256),
             dict(warm_start=1, local_windows=4096, local_maxdeg=8),
             dict(warm_start=1, cap_certify=0), dict(warm_start=1, cap_certify=1, local_windows=0)]


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
@pytest.mark.parametrize("make", [lambda: gen.config(1, 2), lambda: gen.rmat_game(13, 8, seed=4),
                                  lambda: gen.grid_game(40, 40, seed=3),
                                  lambda: gen.varied_game(4000, 2, 16, 3000, seed=8),
                                  lambda: gen.tiny_game(500, max_deg=5, wlo=-5, whi=5, seed=5)],
                         ids=["uniform1k", "rmat13", "grid40", "varied4k", "tiny500"])
def test_schedules_do_not_change_results(make, sched):
    # warm start and local chaining change only the order of lifts
    a = make()
    out, st = gpu(a, 0, **sched)
    np.testing.assert_array_equal(out, ref(a))
    if not sched["warm_start"]:
        assert st.seeded == 0


def test_warm_start_marks_only_losing_vertices():
    a = gen.rmat_game(14, 8, seed=2)
    f = ref(a)
    out, st = gpu(a, 0, warm_start=1)
    np.testing.assert_array_equal(out, f)
    assert 0 < st.seeded <= int((f == TOP64).sum())


def test_warm_start_under_threshold_view():
    a = gen.rmat_game(11, 8, seed=6)
    for k in (-64, 3, 90):
        wq = gen.threshold_weights(a.w, k, 100)
        out, _ = gpu(a, 0, scale=256, shift=k * 100, warm_start=1, local_windows=256)
        np.testing.assert_array_equal(out, ref(a, wq))


def test_option_validation():
    a = gen.config(1, 1)
    with eg.Arena(a) as ar:
        for opt, val in ((99, 1), (eg.EG_OPT_WARM_START, 2), (eg.EG_OPT_LOCAL_WINDOWS, -1),
                         (eg.EG_OPT_CAP_CERTIFY, -1)):
            with pytest.raises(eg.EGError) as ei:
                eg.eg_set_option(ar.handle, opt, val)
            assert ei.value.status == eg.EG_ERR_INVALID


# Certified trial caps: a dual lift proves player-1 wins, a capped lift of the
# game finishes the rest; the result must be the least fixpoint of cap C
# whichever way the trials end (exact at the first cap, after growing it, or
# by the final solve with cap C).
CERT_GAMES = [lambda: gen.grid_game(32, 32, seed=1), lambda: gen.grid_game(48, 80, seed=4),
              lambda: gen.grid_game(96, 96, seed=2), lambda: gen.rmat_game(12, 8, seed=1),
              lambda: gen.varied_game(5000, 2, 16, 1000, seed=3), lambda: gen.uniform_game(1000, 4, -10, 10, 2),
              lambda: gen.tiny_game(300, max_deg=4, wlo=-6, whi=6, seed=9)]


@pytest.mark.parametrize("mult", [16, 4, 1])
@pytest.mark.parametrize("make", CERT_GAMES, ids=["grid32", "grid48x80", "grid96", "rmat12", "varied5k",
                                                 "uniform1k", "tiny300"])
def test_certified_caps_exact(make, mult):
    a = make()
    f = ref(a)
    for bits in (0, 64):
        out, st = gpu(a, bits, cap_certify=mult, certify_after=0)
        np.testing.assert_array_equal(out, f)
        # every vertex the dual lift proves lost is lost
        assert 0 <= st.seeded <= int((f == TOP64).sum())


def test_certified_caps_prove_every_loss_on_grids():
    # at cap 16 max|w| the grid's trials end exact, so the proven set is W1
    a = gen.grid_game(64, 64, seed=1)
    f = ref(a)
    out, st = gpu(a, 64, cap_certify=16, certify_after=0)
    np.testing.assert_array_equal(out, f)
    assert st.seeded == int((f == TOP64).sum())
    _, st_plain = gpu(a, 64, cap_certify=0)
    assert st.relaxations * 20 < st_plain.relaxations
    # the default: a short plain attempt, then the trials
    out, st_def = gpu(a, 64)
    np.testing.assert_array_equal(out, f)
    assert st_def.seeded == int((f == TOP64).sum())


@pytest.mark.parametrize("k", [-128, -3, 0, 2, 100])
def test_certified_caps_under_threshold_view(k):
    a = gen.rmat_game(11, 8, seed=7)
    wq = gen.threshold_weights(a.w, k, 100)
    f = ref(a, wq)
    for mult in (16, 2):
        out, st = gpu(a, 0, scale=256, shift=k * 100, cap_certify=mult, certify_after=0)
        np.testing.assert_array_equal(out, f)
        assert st.seeded <= int((f == TOP64).sum())


def _ominus(a, b, C):
    if a == TOP64:
        return TOP64
    d = int(a) - int(b)
    return TOP64 if d > C else max(0, d)


@pytest.mark.parametrize("make,scale,shift", [
    (lambda: gen.config(1, 3), 1, 0), (lambda: gen.rmat_game(12, 8, seed=2), 1, 0),
    (lambda: gen.grid_game(32, 32, seed=6), 1, 0), (lambda: gen.varied_game(2000, 2, 16, 500, seed=5), 1, 0),
    (lambda: gen.rmat_game(11, 8, seed=8), 256, -300), (lambda: gen.tiny_game(300, 4, -6, 6, seed=3), 1, 0)],
    ids=["uniform1k", "rmat12", "grid32", "varied2k", "rmat11_threshold", "tiny300"])
def test_strategy_attains_the_credits(make, scale, shift):
    # restricting every winning player-0 vertex to its chosen edge must leave
    # every credit unchanged (the oracle solves the restricted game)
    a = make()
    w = np.asarray(a.w, dtype=np.int64) * scale - shift
    f = ref(a, w)
    with eg.Arena(a) as ar:
        out, st = ar.solve(credit_bits=64, w_scale=scale, w_shift=shift)
        np.testing.assert_array_equal(out, f)
        succ = eg.eg_strategy(ar.handle, 64, scale, shift, out)
        import torch
        dev_f = torch.from_numpy(out).cuda()
        dev_s = torch.empty(a.n, dtype=torch.int32, device="cuda")
        eg.eg_strategy(ar.handle, 64, scale, shift, dev_f, dev_s)
        np.testing.assert_array_equal(dev_s.cpu().numpy(), succ)
    C = oracle.bound(a.n, a.row_ptr, w)
    p1 = gen.unpack_owner(a.owner_bits, a.n).astype(bool)
    rp = np.asarray(a.row_ptr, dtype=np.int64)
    rows, ws = [], []
    for v in range(a.n):
        lo, hi = int(rp[v]), int(rp[v + 1])
        if p1[v] or f[v] == TOP64:
            assert succ[v] == -1
            rows.append(list(a.col[lo:hi]))
            ws.append(list(w[lo:hi]))
            continue
        pick = next(e for e in range(lo, hi) if _ominus(f[int(a.col[e])], w[e], C) == f[v])
        assert succ[v] == a.col[pick]
        rows.append([int(a.col[pick])])
        ws.append([int(w[pick])])
    rrp = np.zeros(a.n + 1, dtype=np.int64)
    rrp[1:] = np.cumsum([len(r) for r in rows])
    rcol = np.array([c for r in rows for c in r], dtype=np.int32)
    rw = np.array([x for r in ws for x in r], dtype=np.int64)
    g, _ = oracle.solve(a.n, rrp, rcol, rw, a.owner_bits)
    np.testing.assert_array_equal(g, f)


def test_strategy_rejects_credits_that_are_not_the_least_epm():
    a = gen.config(1, 4)
    with eg.Arena(a) as ar:
        out, _ = ar.solve(credit_bits=64)
        bad = out.copy()
        p1 = gen.unpack_owner(a.owner_bits, a.n).astype(bool)
        v = int(np.nonzero(~p1 & (out != TOP64))[0][0])
        bad[v] += 12345
        with pytest.raises(eg.EGError) as ei:
            eg.eg_strategy(ar.handle, 64, 1, 0, bad)
        assert ei.value.status == eg.EG_ERR_INVALID


def test_cli_solves_and_reports(capsys):
    from paper_1710_03647_gb300 import cli

    cli.main(["--workload", "grid", "--side", "24", "--bits", "64", "--repeat", "2"])
    lines = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert len(lines) == 2 and all(x["status"] == 0 and x["n"] == 576 for x in lines)
    cli.main(["--workload", "rmat", "--scale", "10", "--local-windows", "0", "--max-rounds", "1"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["status"] in (0, eg.EG_ERR_BUDGET) and line["rounds"] <= 1
    cli.main(["--workload", "batch", "--games", "5", "--repeat", "2"])
    lines = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert len(lines) == 2 and all(x["status"] == 0 and x["games"] == 5 for x in lines)
    assert lines[0]["relaxations"] > 0
