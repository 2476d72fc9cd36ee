"""GPU tests of the failure paths, made on the host without faulting the GPU:

* a grid-barrier wait that runs out: a wait limit of 1 microsecond makes the
  ordinary waits of a persistent solve expire; the solve must end with
  EG_ERR_TIMEOUT (every block leaves at its next barrier), leave credits at
  or below the least fixpoint, and the same arena must then solve
  bit-exactly against the oracle with the limit restored;
* a round budget that runs out inside the certified trials;
* admission that finds no pool room: the server's test hook makes the next
  reservations fail; the request must stay queued, be admitted on a retry
  and give the oracle's credits.
"""
from __future__ import annotations

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


def exact(a):
    f, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
    return f


def below_or_equal(got, want):
    """got <= want elementwise in the order of Sec. 3.1 (TOP the largest)."""
    return bool(np.all(got <= want))


def test_wait_limit_runs_out_then_arena_solves_again():
    a = gen.grid_game(128, 128, seed=3)
    want = exact(a)
    with eg.Arena(a) as ar:
        ar.tune(wait_limit_us=1)
        timeouts = 0
        for _ in range(5):
            out = np.full(a.n, -1, dtype=np.int64)
            rc, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out, raise_on_error=False)
            assert rc in (eg.EG_OK, eg.EG_ERR_TIMEOUT), eg.eg_last_error()
            assert st.status == rc
            if rc == eg.EG_OK:
                np.testing.assert_array_equal(out, want)
                continue
            timeouts += 1
            assert "limit" in eg.eg_last_error()
            assert (out >= 0).all() and below_or_equal(out, want)
        assert timeouts > 0, "a 1 us barrier wait never ran out"
        ar.tune(wait_limit_us=5_000_000)
        out = np.empty(a.n, dtype=np.int64)
        _, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out)
        assert st.status == eg.EG_OK
        np.testing.assert_array_equal(out, want)


def test_wait_limit_runs_out_in_a_plan():
    gs = [gen.grid_game(64, 64, seed=s) for s in (1, 2)]
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(gs)
    h = eg.eg_create(n, int(row_ptr[-1]), row_ptr, col, w, owner_bits=owner_bits)
    try:
        eg.eg_set_parts(h, part_ptr)
        wants = np.concatenate([exact(g) for g in gs])
        with eg.Plan(h, len(gs)) as plan:
            eg.eg_set_option(h, eg.EG_OPT_WAIT_LIMIT_US, 1)
            seen = set()
            for _ in range(5):
                out, st = plan.run(raise_on_error=False)
                seen.add(st.status)
                assert st.status in (eg.EG_OK, eg.EG_ERR_TIMEOUT)
                assert below_or_equal(out, wants) and (out >= 0).all()
            assert eg.EG_ERR_TIMEOUT in seen
            eg.eg_set_option(h, eg.EG_OPT_WAIT_LIMIT_US, 5_000_000)
            out, st = plan.run()
            np.testing.assert_array_equal(out, wants)
    finally:
        eg.eg_destroy(h)


@pytest.mark.parametrize("rounds", [1, 3, 9, 20])
def test_budget_inside_the_trials_stays_below_the_fixpoint(rounds):
    a = gen.grid_game(256, 256, seed=1)
    want = exact(a)
    with eg.Arena(a) as ar:
        ar.tune(certify_after=2)  # the trials start after 2 rounds
        out = np.full(a.n, -1, dtype=np.int64)
        rc, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out, max_rounds=rounds, raise_on_error=False)
        if rc == eg.EG_OK:
            np.testing.assert_array_equal(out, want)
        else:
            assert rc == eg.EG_ERR_BUDGET and st.status == rc
            assert (out >= 0).all() and below_or_equal(out, want)
        # the arena is clean for the next solve
        _, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out)
        np.testing.assert_array_equal(out, want)


def _wait(server, ticket, out, timeout=60.0):
    t0 = time.time()
    while True:
        rc, st = eg.eg_poll(server, ticket, out)
        if rc != eg.EG_PENDING:
            return rc, st
        assert time.time() - t0 < timeout
        time.sleep(0.001)


def test_admission_refuses_then_retries():
    gs = [gen.config(1, 1), gen.varied_game(3000, 2, 16, 500, seed=4), gen.grid_game(30, 30, seed=5)]
    arenas = [eg.Arena(g) for g in gs]
    server = eg.eg_server_create(1 << 30, 4)
    try:
        eg.eg_server_set_option(server, eg.EG_SRV_IDLE_SOLO, 0)  # every request goes to the pool
        eg.eg_server_set_option(server, eg.EG_SRV_FAIL_RESERVATIONS, 3)
        tickets = [eg.eg_submit(server, a.handle, 0, 1, 0) for a in arenas]
        for g, t in zip(gs, tickets):
            out = np.empty(g.n, dtype=np.int64)
            rc, _ = _wait(server, t, out)
            assert rc == eg.EG_OK, eg.eg_last_error()
            np.testing.assert_array_equal(out, exact(g))
        c = eg.eg_server_counters_get(server)
        assert c["refused"] >= 3
        assert c["submitted"] == 3 and c["completed"] == 3 and c["admitted"] == 3
        with pytest.raises(eg.EGError):
            eg.eg_server_set_option(server, 99, 1)
    finally:
        eg.eg_server_destroy(server)
        for a in arenas:
            a.close()
