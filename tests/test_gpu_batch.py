"""GPU parity of batched solves (eg_plan): every instance of a batch equals
the CPU oracle on that game and weight map alone, for uneven game sizes and
for many threshold queries sharing one arena."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen
from tests._games import TOP64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def ref(a, w=None):
    f, _ = oracle.solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)
    return f


def packed_arena(games):
    n, rp, col, w, ob, pp = eg.pack_games(games)
    h = eg.eg_create(n, int(rp[-1]), rp, col, w, owner_bits=ob)
    eg.eg_set_parts(h, pp)
    return h


def mixed_games():
    gs = [gen.uniform_game(700 + 37 * k, 4, -10, 10, seed=k) for k in range(3)]
    gs += [gen.varied_game(1500 + 200 * k, 2, 16, 10 ** (1 + k), seed=50 + k) for k in range(3)]
    gs += [gen.rmat_game(11, 8, seed=7), gen.grid_game(20, 30, seed=4), gen.tiny_game(9, 3, -3, 3, seed=2)]
    return gs


@pytest.mark.parametrize("warm", [0, 1])
@pytest.mark.parametrize("bits", [0, 64])
def test_batch_of_uneven_games(warm, bits):
    games = mixed_games()
    h = packed_arena(games)
    try:
        eg.eg_set_option(h, eg.EG_OPT_WARM_START, warm)
        with eg.Plan(h, len(games), credit_bits=bits) as plan:
            out, st = plan.run()
            for k, g in enumerate(games):
                off, n, C, b = plan.instance(k)
                assert n == g.n and C == oracle.bound(g.n, g.row_ptr, g.w)
                np.testing.assert_array_equal(out[off:off + n], ref(g))
            again, _ = plan.run()  # graph replay
            np.testing.assert_array_equal(again, out)
    finally:
        eg.eg_destroy(h)


def test_batch_subset_and_repeats():
    games = mixed_games()
    h = packed_arena(games)
    try:
        part = [3, 3, 0, 7, 1]
        with eg.Plan(h, len(part), part=part) as plan:
            out, _ = plan.run()
            for i, k in enumerate(part):
                off, n, _, _ = plan.instance(i)
                np.testing.assert_array_equal(out[off:off + n], ref(games[k]))
    finally:
        eg.eg_destroy(h)


def test_threshold_queries_share_one_arena():
    a = gen.rmat_game(12, 8, seed=3)
    W = 100
    ks = [-128, -40, -3, 0, 1, 2, 7, 30, 127]
    h = eg.eg_create(a.n, a.m, a.row_ptr, a.col, a.w, owner_bits=a.owner_bits)
    try:
        with eg.Plan(h, len(ks), part=[0] * len(ks), w_scale=[256] * len(ks),
                     w_shift=[k * W for k in ks]) as plan:
            out, st = plan.run()
            for i, k in enumerate(ks):
                off, n, C, _ = plan.instance(i)
                wq = gen.threshold_weights(a.w, k, W)
                assert C == oracle.bound(a.n, a.row_ptr, wq)
                np.testing.assert_array_equal(out[off:off + n], ref(a, wq))
    finally:
        eg.eg_destroy(h)


def test_batch_matches_single_solves_device_output():
    torch = pytest.importorskip("torch")
    games = mixed_games()[:5]
    h = packed_arena(games)
    try:
        with eg.Plan(h, len(games), credit_bits=64) as plan:
            dev = torch.empty(plan.total, dtype=torch.int64, device="cuda:0")
            plan.run(dev)
            got = dev.cpu().numpy()
            for k, g in enumerate(games):
                off, n, _, _ = plan.instance(k)
                with eg.Arena(g) as single:
                    alone, _ = single.solve(64)
                np.testing.assert_array_equal(got[off:off + n], alone)
    finally:
        eg.eg_destroy(h)


def test_batch_int32_overflow_and_bad_parts():
    big = gen.Arena(3, np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 2], np.int32),
                    np.array([-2 ** 30, -2 ** 30, 0], np.int32), gen.pack_owner(np.array([1, 1, 0], bool)))
    games = [gen.config(1, 1), big]
    h = packed_arena(games)
    try:
        with pytest.raises(eg.EGError) as ei:
            eg.Plan(h, 2, credit_bits=32)
        assert ei.value.status == eg.EG_ERR_OVERFLOW
        with eg.Plan(h, 2) as plan:
            out, st = plan.run()
            assert st.credit_bits == 64
            assert plan.instance(0)[3] == 32 and plan.instance(1)[3] == 64
            off, n, _, _ = plan.instance(1)
            np.testing.assert_array_equal(out[off:off + n], ref(big))
        with pytest.raises(eg.EGError) as ei:
            eg.eg_set_parts(h, [0, 500, 1003])  # cuts game 0 in two
        assert ei.value.status == eg.EG_ERR_INVALID
    finally:
        eg.eg_destroy(h)


def test_batch_round_budget_then_run():
    games = mixed_games()[:4]
    h = packed_arena(games)
    try:
        eg.eg_set_option(h, eg.EG_OPT_WARM_START, 0)
        eg.eg_set_option(h, eg.EG_OPT_LOCAL_WINDOWS, 0)
        with eg.Plan(h, len(games)) as plan:
            _, st = plan.run(max_rounds=2, raise_on_error=False)
            assert st.status == eg.EG_ERR_BUDGET
            out, _ = plan.run()
            for k, g in enumerate(games):
                off, n, _, _ = plan.instance(k)
                np.testing.assert_array_equal(out[off:off + n], ref(g))
    finally:
        eg.eg_destroy(h)


@pytest.mark.parametrize("after", [64, 0, 3])
@pytest.mark.parametrize("mult", [4, 1])
def test_batch_certified_trials_per_instance(after, mult):
    # grids need the certified trials; the small games finish in the first
    # attempt (after > 0) and must stay as they are through the later trials
    games = [gen.grid_game(40, 40, seed=3), gen.grid_game(24, 50, seed=8), gen.config(1, 5),
             gen.rmat_game(10, 8, seed=9), gen.varied_game(2500, 2, 16, 5000, seed=12),
             gen.tiny_game(7, 3, -3, 3, seed=4)]
    h = packed_arena(games)
    try:
        eg.eg_set_option(h, eg.EG_OPT_CAP_CERTIFY, mult)
        eg.eg_set_option(h, eg.EG_OPT_CERTIFY_AFTER, after)
        with eg.Plan(h, len(games)) as plan:
            out, st = plan.run()
            for k, g in enumerate(games):
                off, n, _, _ = plan.instance(k)
                np.testing.assert_array_equal(out[off:off + n], ref(g))
            again, _ = plan.run()
            np.testing.assert_array_equal(again, out)
    finally:
        eg.eg_destroy(h)


def test_threshold_batch_certified_against_oracle():
    a = gen.rmat_game(12, 8, seed=21)
    ks = [-100, -20, -3, -1, 0, 1, 2, 5, 40, 127]
    W = 100
    h = eg.eg_create(a.n, a.m, a.row_ptr, a.col, a.w, owner_bits=a.owner_bits)
    try:
        with eg.Plan(h, len(ks), part=[0] * len(ks), w_scale=[256] * len(ks), w_shift=[k * W for k in ks]) as plan:
            out, _ = plan.run()
            for i, k in enumerate(ks):
                off, n, _, _ = plan.instance(i)
                np.testing.assert_array_equal(out[off:off + n], ref(a, gen.threshold_weights(a.w, k, W)))
    finally:
        eg.eg_destroy(h)
