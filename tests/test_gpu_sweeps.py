"""GPU tests of two launch settings that must not change a result
(Sec. 3.1: the least fixpoint does not depend on the order of the lifts):

* EG_OPT_SWEEPS -- dense in-place sweeps of every credit before the worklist
  rounds, the last one seeding the first round's push list;
* EG_OPT_CHUNK_EDGES -- long worklists worked in fixed-size chunks that the
  warps take in list order instead of one piece per warp.

Each setting is checked element by element against the oracle on the plain
route (cap C, Algorithm 1's fixpoint), the certified route (dual and capped
trials, which also run the sweeps and chunks), int32 and int64 credits,
threshold views, batched plans, and at full size on the R-MAT scale-18 arena
against its stored oracle digest.  Small chunk sizes force the chunked split
on these sizes (it starts once a list holds more than chunk edges per warp).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen
from tests._games import GOLDEN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def plain(a, w=None):
    f, _ = oracle.solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)
    return f


def certified(a, w=None):
    f, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)
    return f


GAMES = {
    "uniform1k": (lambda: gen.config(1, seed=2), plain),
    "rmat12": (lambda: gen.rmat_game(12, 8, seed=3), plain),
    "varied": (lambda: gen.varied_game(5000, 2, 9, 300, seed=5), certified),
    "grid120": (lambda: gen.grid_game(120, 120, seed=6), certified),
    "grid64x150": (lambda: gen.grid_game(64, 150, seed=7), certified),
}


@pytest.mark.parametrize("sweeps", [1, 2, 5])
@pytest.mark.parametrize("name", list(GAMES))
def test_sweeps_keep_the_oracle_credits(name, sweeps):
    make, ref = GAMES[name]
    a = make()
    want = ref(a)
    with eg.Arena(a) as ar:
        for route in ({}, {"certify_after": 0}, {"warm_start": 0}):
            opts = dict(sweeps=sweeps, warm_start=1, certify_after=8)
            opts.update(route)
            ar.tune(**opts)
            for bits in (0, 64):
                out, st = ar.solve(credit_bits=bits)
                assert st.status == eg.EG_OK, (route, bits)
                np.testing.assert_array_equal(out, want, err_msg=f"{route} bits={bits}")


def test_sweeps_count_their_relaxations():
    a = gen.varied_game(6000, 2, 9, 100, seed=8)
    want = certified(a)
    with eg.Arena(a) as ar:
        ar.tune(sweeps=0)
        out0, st0 = ar.solve(64)
        ar.tune(sweeps=6)
        out6, st6 = ar.solve(64)
    np.testing.assert_array_equal(out0, want)
    np.testing.assert_array_equal(out6, want)
    # the first sweep alone evaluates every edge of every credit not seeded at TOP
    assert st6.relaxations >= int(a.row_ptr[-1]) // 2
    assert st6.rounds >= 0


@pytest.mark.parametrize("chunk", [32, 96, 1000])
@pytest.mark.parametrize("name", list(GAMES))
def test_chunked_lists_keep_the_oracle_credits(name, chunk):
    make, ref = GAMES[name]
    a = make()
    want = ref(a)
    with eg.Arena(a) as ar:
        for route in ({}, {"certify_after": 0}):
            ar.tune(chunk_edges=chunk, local_windows=0, **route)
            for bits in (0, 64):
                out, st = ar.solve(credit_bits=bits)
                assert st.status == eg.EG_OK
                np.testing.assert_array_equal(out, want, err_msg=f"{route} bits={bits}")


@pytest.mark.parametrize("k", [-40, 0, 50])
def test_sweeps_and_chunks_under_threshold_views(k):
    a = gen.grid_game(90, 90, seed=4)
    w2 = gen.threshold_weights(a.w, k, 10, scale=4)
    want = certified(a, w2)
    with eg.Arena(a) as ar:
        ar.tune(sweeps=3, chunk_edges=32)
        for bits in (0, 64):
            out, _ = ar.solve(credit_bits=bits, w_scale=4, w_shift=k * 10)
            np.testing.assert_array_equal(out, want)


@pytest.mark.parametrize("sweeps,chunk", [(0, 32), (2, 1024), (4, 64)])
def test_plans_with_sweeps_and_chunks(sweeps, chunk):
    games = [gen.varied_game(n, 2, 8, W, seed=20 + i) for i, (n, W) in
             enumerate([(1500, 50), (4000, 400), (900, 3000), (6000, 20), (2500, 800), (3000, 100)])]
    wants = [certified(g) for g in games]
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(games)
    h = eg.eg_create(n, int(row_ptr[-1]), row_ptr, col, w, owner_bits=owner_bits)
    try:
        eg.eg_set_parts(h, part_ptr)
        eg.eg_set_option(h, eg.EG_OPT_SWEEPS, sweeps)
        eg.eg_set_option(h, eg.EG_OPT_CHUNK_EDGES, chunk)
        for certify_after in (8, 0):
            eg.eg_set_option(h, eg.EG_OPT_CERTIFY_AFTER, certify_after)
            with eg.Plan(h, len(games)) as plan:
                for _ in range(2):  # the second run replays the captured graph
                    out, st = plan.run()
                    assert st.status == eg.EG_OK
                    for i, want in enumerate(wants):
                        off, gn, _, _ = plan.instance(i)
                        np.testing.assert_array_equal(out[off:off + gn], want, err_msg=f"game {i}")
    finally:
        eg.eg_destroy(h)


def test_rmat18_full_size_with_sweeps_and_chunks_against_stored_oracle():
    g = json.load(open(os.path.join(GOLDEN, "rmat18_s1.json")))
    a = gen.rmat_game(18, 8, seed=1)
    with eg.Arena(a) as ar:
        for sweeps, chunk in ((3, 64), (0, 32), (8, 1024)):
            ar.tune(sweeps=sweeps, chunk_edges=chunk)
            out, st = ar.solve(credit_bits=64)
            assert st.status == eg.EG_OK and st.C == g["C"]
            got = hashlib.sha256(np.ascontiguousarray(out, dtype=np.int64).tobytes()).hexdigest()
            assert got == g["sha256"], (sweeps, chunk)


def test_option_ranges():
    a = gen.config(1, seed=1)
    with eg.Arena(a) as ar:
        with pytest.raises(eg.EGError):
            eg.eg_set_option(ar.handle, eg.EG_OPT_SWEEPS, 1025)
        with pytest.raises(eg.EGError):
            eg.eg_set_option(ar.handle, eg.EG_OPT_CHUNK_EDGES, -1)
        eg.eg_set_option(ar.handle, eg.EG_OPT_SWEEPS, 0)
        eg.eg_set_option(ar.handle, eg.EG_OPT_CHUNK_EDGES, 0)
