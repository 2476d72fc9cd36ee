"""GPU tests of the request loop (eg_server_create / eg_submit / eg_poll):
every request's credits are the same alone and in the mix, including
requests submitted from several threads while earlier batches run."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def wait(server, ticket, out=None, timeout=60.0):
    t0 = time.time()
    while True:
        rc, st = eg.eg_poll(server, ticket, out)
        if rc != eg.EG_PENDING:
            return rc, st
        if time.time() - t0 > timeout:
            raise TimeoutError(ticket)
        time.sleep(0.001)


def alone(handle, bits, scale, shift, n):
    out = np.empty(n, dtype=np.int32 if bits == 32 else np.int64)
    eg.eg_solve_credit(handle, bits, scale, shift, out)
    return out


def games():
    return [gen.config(1, 1), gen.varied_game(3000, 2, 16, 500, seed=4), gen.rmat_game(12, 8, seed=2),
            gen.grid_game(30, 30, seed=5), gen.tiny_game(40, 4, -3, 3, seed=9), gen.uniform_game(5000, 3, -20, 20, 6)]


def test_mix_equals_alone():
    gs = games()
    arenas = [eg.Arena(g) for g in gs]
    maps = lambda i: ((0, 1, 0), (32, 1, 0), (64, 256, (i - 2) * 100))  # noqa: E731
    # each arena solved alone first: no arena is solved by the caller while
    # a request for it is pending
    want = {(i, m): alone(a.handle, *m, gs[i].n) for i, a in enumerate(arenas) for m in maps(i)}
    server = eg.eg_server_create(8 << 30, 16)
    try:
        reqs = []
        for i, (g, a) in enumerate(zip(gs, arenas)):
            for m in maps(i):
                reqs.append((i, m, eg.eg_submit(server, a.handle, *m)))
        for i, m, t in reqs:
            out = np.empty(gs[i].n, dtype=np.int32 if m[0] == 32 else np.int64)
            rc, st = wait(server, t, out)
            assert rc == eg.EG_OK, (i, m, rc, eg.eg_last_error())
            np.testing.assert_array_equal(out, want[(i, m)])
            assert st.ms > 0
        # one more check against the oracle itself
        f, _ = oracle.solve(gs[2].n, gs[2].row_ptr, gs[2].col, gs[2].w, gs[2].owner_bits)
        t = eg.eg_submit(server, arenas[2].handle, 0, 1, 0)
        out = np.empty(gs[2].n, dtype=np.int64)
        assert wait(server, t, out)[0] == eg.EG_OK
        np.testing.assert_array_equal(out, f)
    finally:
        eg.eg_server_destroy(server)
        for a in arenas:
            a.close()


def test_arrivals_from_threads_while_batches_run():
    gs = games()
    arenas = [eg.Arena(g) for g in gs]
    want = {i: alone(a.handle, 0, 1, 0, g.n) for i, (g, a) in enumerate(zip(gs, arenas))}
    server = eg.eg_server_create(8 << 30, 4)  # 4 slots: later arrivals wait for a free slot
    got, errors = [], []

    def client(seed):
        rng = np.random.default_rng(seed)
        mine = []
        for _ in range(12):
            i = int(rng.integers(len(gs)))
            mine.append((i, eg.eg_submit(server, arenas[i].handle, 0, 1, 0)))
            time.sleep(float(rng.random()) * 0.003)
        for i, t in mine:
            out = np.empty(gs[i].n, dtype=np.int64)
            rc, _ = wait(server, t, out)
            if rc != eg.EG_OK:
                errors.append((i, rc))
            got.append((i, out))

    try:
        ths = [threading.Thread(target=client, args=(s,)) for s in range(3)]
        for t in ths:
            t.start()
        for t in ths:
            t.join(timeout=120)
        assert not errors
        assert len(got) == 36
        for i, out in got:
            np.testing.assert_array_equal(out, want[i])
    finally:
        eg.eg_server_destroy(server)
        for a in arenas:
            a.close()


def test_budget_and_errors():
    small, big = gen.config(1, 3), gen.rmat_game(14, 8, seed=1)
    a_small, a_big = eg.Arena(small), eg.Arena(big)
    want = alone(a_small.handle, 0, 1, 0, small.n)
    server = eg.eg_server_create(1 << 20, 8)  # 1 MiB: the small game fits, the big one does not
    try:
        t_big = eg.eg_submit(server, a_big.handle, 0, 1, 0)
        t_small = eg.eg_submit(server, a_small.handle, 0, 1, 0)
        out = np.empty(small.n, dtype=np.int64)
        assert wait(server, t_small, out)[0] == eg.EG_OK
        np.testing.assert_array_equal(out, want)
        assert wait(server, t_big)[0] == eg.EG_ERR_OOM
        rc, _ = eg.eg_poll(server, 987654321)
        assert rc == eg.EG_ERR_INVALID
        with pytest.raises(eg.EGError):
            eg.eg_submit(server, a_small.handle, 16, 1, 0)
    finally:
        eg.eg_server_destroy(server)
        a_small.close()
        a_big.close()


def test_destroy_with_pending_requests():
    g = gen.rmat_game(13, 8, seed=3)
    a = eg.Arena(g)
    server = eg.eg_server_create(4 << 30, 2)
    for _ in range(20):
        eg.eg_submit(server, a.handle, 0, 1, 0)
    eg.eg_server_destroy(server)  # returns after the running batch; queued ones are dropped
    a.close()


def test_late_arrivals_join_the_running_solve():
    # a slow game (a 64 x 64 grid without certified caps takes thousands of
    # rounds, and certification is off for it here) is being solved when small games arrive: they join the
    # resident solve at its next round and finish while the slow one runs,
    # and every result equals the solve of that game alone
    slow = gen.grid_game(64, 64, seed=1)
    smalls = [gen.config(1, s) for s in (2, 3, 4)] + [gen.rmat_game(10, 8, seed=5)]
    a_slow = eg.Arena(slow)
    a_slow.tune(cap_certify=0)  # keep it in the resident solve (no certified take-over)
    a_small = [eg.Arena(g) for g in smalls]
    want_small = [alone(a.handle, 0, 1, 0, g.n) for g, a in zip(smalls, a_small)]
    want_slow = alone(a_slow.handle, 64, 1, 0, slow.n)
    server = eg.eg_server_create(2 << 30, 8)
    try:
        t_slow = eg.eg_submit(server, a_slow.handle, 64, 1, 0)
        time.sleep(0.05)
        ts = [eg.eg_submit(server, a.handle, 0, 1, 0) for a in a_small]
        for g, want, t in zip(smalls, want_small, ts):
            out = np.empty(g.n, dtype=np.int64)
            rc, st = wait(server, t, out)
            assert rc == eg.EG_OK, eg.eg_last_error()
            np.testing.assert_array_equal(out, want)
        rc, _ = eg.eg_poll(server, t_slow)
        assert rc == eg.EG_PENDING  # the small games did not wait for it
        out = np.empty(slow.n, dtype=np.int64)
        rc, st = wait(server, t_slow, out, timeout=120)
        assert rc == eg.EG_OK
        np.testing.assert_array_equal(out, want_slow)
        assert st.rounds > 0 and st.fixpoint_ms > 0
    finally:
        eg.eg_server_destroy(server)
        a_slow.close()
        for a in a_small:
            a.close()


def test_slow_games_are_taken_out_to_the_certified_route():
    # grids stay unfinished past EG_OPT_CERTIFY_AFTER rounds in the resident
    # solve; the server solves them alone with certified trial caps, retires
    # their slots, and keeps serving the others
    hard = [gen.grid_game(48, 48, seed=2), gen.grid_game(40, 64, seed=5)]
    easy = [gen.config(1, 7), gen.rmat_game(11, 8, seed=3)]
    games = hard + easy
    arenas = [eg.Arena(g) for g in games]
    want = [alone(a.handle, 0, 1, 0, g.n) for g, a in zip(games, arenas)]
    server = eg.eg_server_create(1 << 30, 4)
    try:
        for rep in range(2):  # the second pass reuses slots freed by retirement
            ts = [eg.eg_submit(server, a.handle, 0, 1, 0) for a in arenas]
            for i, t in enumerate(ts):
                out = np.empty(games[i].n, dtype=np.int64)
                rc, st = wait(server, t, out, timeout=120)
                assert rc == eg.EG_OK, eg.eg_last_error()
                np.testing.assert_array_equal(out, want[i])
                if i < len(hard):
                    assert st.seeded > 0  # proven player-1 vertices: the certified route ran
    finally:
        eg.eg_server_destroy(server)
        for a in arenas:
            a.close()


def test_large_games_are_solved_alone_between_slices():
    # a game of at least 2^19 edges skips the pool and is solved alone between
    # resident slices; its credits (each width) equal the solve of it alone,
    # and the small games in the mix are unaffected
    big = gen.rmat_game(17, 8, seed=4)
    assert big.m >= 1 << 19
    smalls = [gen.config(1, 5), gen.rmat_game(12, 8, seed=6), gen.grid_game(24, 24, seed=3)]
    games = [big] + smalls
    arenas = [eg.Arena(g) for g in games]
    maps = ((0, 1, 0), (32, 1, 0), (64, 4, 7))
    want = {(i, m): alone(a.handle, *m, games[i].n) for i, a in enumerate(arenas) for m in maps}
    server = eg.eg_server_create(4 << 30, 8)
    try:
        reqs = []
        for i, a in enumerate(arenas):
            for m in maps:
                reqs.append((i, m, eg.eg_submit(server, a.handle, *m)))
        for i, m, t in reqs:
            out = np.empty(games[i].n, dtype=np.int32 if m[0] == 32 else np.int64)
            rc, st = wait(server, t, out, timeout=120)
            assert rc == eg.EG_OK, (i, m, rc, eg.eg_last_error())
            np.testing.assert_array_equal(out, want[(i, m)])
            assert st.ms > 0
    finally:
        eg.eg_server_destroy(server)
        for a in arenas:
            a.close()


def test_idle_server_answers_a_lone_request_alone():
    # a request that finds the server idle gets a short attempt by the
    # single-game route; a game that attempt does not finish joins the pool
    easy = gen.rmat_game(12, 8, seed=9)
    slow = gen.grid_game(64, 64, seed=1)
    a_easy, a_slow = eg.Arena(easy), eg.Arena(slow)
    a_slow.tune(cap_certify=0)  # stays in the resident solve once admitted
    want_easy = alone(a_easy.handle, 0, 1, 0, easy.n)
    want_slow = alone(a_slow.handle, 64, 1, 0, slow.n)
    server = eg.eg_server_create(1 << 30, 4)
    try:
        out = np.empty(easy.n, dtype=np.int64)
        rc, st = wait(server, eg.eg_submit(server, a_easy.handle, 0, 1, 0), out)
        assert rc == eg.EG_OK
        np.testing.assert_array_equal(out, want_easy)
        c = eg.eg_server_counters_get(server)
        assert c["idle_solo"] == 1 and c["admitted"] == 0
        out = np.empty(slow.n, dtype=np.int64)
        rc, st = wait(server, eg.eg_submit(server, a_slow.handle, 64, 1, 0), out, timeout=120)
        assert rc == eg.EG_OK
        np.testing.assert_array_equal(out, want_slow)
        c = eg.eg_server_counters_get(server)
        assert c["idle_solo"] == 1 and c["admitted"] == 1 and c["completed"] == 2
        eg.eg_server_set_option(server, eg.EG_SRV_IDLE_SOLO, 0)
        out = np.empty(easy.n, dtype=np.int64)
        rc, _ = wait(server, eg.eg_submit(server, a_easy.handle, 0, 1, 0), out)
        assert rc == eg.EG_OK and eg.eg_server_counters_get(server)["admitted"] == 2
        np.testing.assert_array_equal(out, want_easy)
        with pytest.raises(eg.EGError):
            eg.eg_server_set_option(server, eg.EG_SRV_IDLE_SOLO, 2)
    finally:
        eg.eg_server_destroy(server)
        a_easy.close()
        a_slow.close()
