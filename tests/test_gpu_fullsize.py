"""GPU parity at the full sizes of the benchmark workloads, against results
the CPU oracle stored (tests/golden/*.json, written by make_golden.py, which
calls only oracle/ and the input generators).

* the 4000 x 4000 road-like grid (16M vertices, 64.6M edges, int64 credits):
  the oracle's certified composition of capped Algorithm 1 runs decided it;
* the 4096-game uneven batch, solved in one plan: 32 of its games, spread
  over its size range, against their stored credits;
* 256 threshold queries on the R-MAT scale-20 arena in one plan: the queries
  k = -128, 0 and 127 against their stored credits.

Each comparison is of the SHA-256 of the int64 credit array (TOP = INT64_MAX),
i.e. bit-exact.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen
from tests._games import GOLDEN, TOP64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def golden(name):
    return json.load(open(os.path.join(GOLDEN, f"{name}.json")))


def digest(f):
    return hashlib.sha256(np.ascontiguousarray(f, dtype=np.int64).tobytes()).hexdigest()


def test_road_grid_full_size_against_stored_oracle():
    g = golden("grid4000_s1")
    a = gen.config(3, 1)
    with eg.Arena(a) as ar:
        out, st = ar.solve(credit_bits=64)
    assert st.status == eg.EG_OK and st.credit_bits == 64 and st.C == g["C"]
    assert digest(out) == g["sha256"]
    assert int((out == TOP64).sum()) == g["top"]
    # and every lift equation holds (an independent check by the oracle)
    assert oracle.check(a.n, a.row_ptr, a.col, a.w, a.owner_bits, out, st.C)[0] == 0


def test_batch_of_4096_games_sampled_against_stored_oracle():
    g = golden("batch4096_sample")
    games = gen.batch_games(g["count"])
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(games)
    del games
    h = eg.eg_create(n, int(row_ptr[-1]), row_ptr, col, w, owner_bits=owner_bits)
    del col, w
    try:
        eg.eg_set_parts(h, part_ptr)
        with eg.Plan(h, g["count"]) as plan:
            out, st = plan.run()
            assert st.status == eg.EG_OK
            for rec in g["games"]:
                off, gn, C, _ = plan.instance(rec["index"])
                assert gn == rec["n"] and C == rec["C"], rec["index"]
                assert digest(out[off:off + gn]) == rec["sha256"], rec["index"]
    finally:
        eg.eg_destroy(h)


def test_256_threshold_queries_sampled_against_stored_oracle():
    g = golden("thresholds_rmat20")
    a = gen.config(2, 1)
    ks = list(range(-128, 128))
    with eg.Arena(a) as ar:
        with eg.Plan(ar.handle, len(ks), part=[0] * len(ks), w_scale=[256] * len(ks),
                     w_shift=[k * g["W"] for k in ks]) as plan:
            out, st = plan.run()
            assert st.status == eg.EG_OK
            for q in g["queries"]:
                off, qn, C, _ = plan.instance(ks.index(q["k"]))
                assert qn == a.n and C == q["C"]
                assert digest(out[off:off + qn]) == q["sha256"], q["k"]
