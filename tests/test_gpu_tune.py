"""GPU tests of the autotuner (eg_autotune, eg_plan_autotune): the settings
it picks still give the oracle's credits, the choice is cached under the
instance's signature and taken from the cache without timing, and games of
one shape share a signature."""
from __future__ import annotations

import json

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


def exact(a, w=None):
    f, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)
    return f


@pytest.mark.parametrize("make,bits", [(lambda: gen.grid_game(128, 128, seed=4), 64),
                                       (lambda: gen.rmat_game(14, 8, seed=5), 32)], ids=["grid128", "rmat14"])
def test_tuned_settings_keep_the_oracle_credits_and_are_cached(tmp_path, make, bits):
    a = make()
    want = exact(a)
    cache = str(tmp_path / "plans.jsonl")
    with eg.Arena(a) as ar:
        t = eg.eg_autotune(ar.handle, bits, 1, 0, cache, max_solves=40)
        assert t["from_cache"] == 0 and 0 < t["solves"] <= 40
        assert t["tuned_ms"] <= t["default_ms"] * 1.0001
        out, st = ar.solve(credit_bits=bits)
        got = np.where(out == eg.EG_TOP32, oracle.TOP, out.astype(np.int64)) if bits == 32 else out
        np.testing.assert_array_equal(got, want)
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["key"] == t["key"]
    assert lines[0]["local_windows"] == t["local_windows"]
    # a fresh arena of the same game: the settings come from the cache
    with eg.Arena(a) as ar2:
        t2 = eg.eg_autotune(ar2.handle, bits, 1, 0, cache)
        assert t2["from_cache"] == 1 and t2["solves"] == 0 and t2["key"] == t["key"]
        for k in ("local_windows", "local_maxdeg", "blocks_per_sm", "cap_certify", "certify_after", "dual_k", "kick_rounds"):
            assert t2[k] == t[k], k
        out, _ = ar2.solve(credit_bits=bits)
        got = np.where(out == eg.EG_TOP32, oracle.TOP, out.astype(np.int64)) if bits == 32 else out
        np.testing.assert_array_equal(got, want)


def test_signature_is_shared_by_games_of_one_shape(tmp_path):
    cache = str(tmp_path / "plans.jsonl")
    a1, a2 = gen.grid_game(96, 96, seed=1), gen.grid_game(96, 96, seed=2)
    with eg.Arena(a1) as h1, eg.Arena(a2) as h2:
        t1 = eg.eg_autotune(h1.handle, 64, 1, 0, cache, max_solves=12)
        t2 = eg.eg_autotune(h2.handle, 64, 1, 0, cache)
        assert t2["key"] == t1["key"] and t2["from_cache"] == 1
        np.testing.assert_array_equal(h2.solve(64)[0], exact(a2))
    with eg.Arena(gen.rmat_game(12, 8, seed=1)) as h3:
        t3 = eg.eg_autotune(h3.handle, 64, 1, 0, cache, max_solves=8)
        assert t3["key"] != t1["key"] and t3["from_cache"] == 0
    assert len(open(cache).read().splitlines()) == 2


def test_plan_autotune_keeps_every_instance_exact(tmp_path):
    games = [gen.grid_game(40, 40, seed=s) for s in (1, 2)] + [gen.varied_game(2000, 2, 16, 300, seed=3),
                                                               gen.rmat_game(11, 8, seed=7)]
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(games)
    h = eg.eg_create(n, int(row_ptr[-1]), row_ptr, col, w, owner_bits=owner_bits)
    try:
        eg.eg_set_parts(h, part_ptr)
        with eg.Plan(h, len(games)) as plan:
            t = eg.eg_plan_autotune(plan, str(tmp_path / "p.jsonl"), max_solves=24)
            assert t["key"].startswith("plan4-") and t["solves"] > 0
            out, st = plan.run()
            assert st.status == eg.EG_OK
            for i, g in enumerate(games):
                off, gn, _, _ = plan.instance(i)
                np.testing.assert_array_equal(out[off:off + gn], exact(g), err_msg=f"game {i}")
    finally:
        eg.eg_destroy(h)


def test_autotune_rejects_bad_arguments():
    with eg.Arena(gen.config(1, 1)) as ar:
        with pytest.raises(eg.EGError):
            eg.eg_autotune(ar.handle, 16)
        with pytest.raises(eg.EGError):
            eg.eg_autotune(ar.handle, 0, 1, 0, None, -1)
