"""GPU tests of the cycle jumps of the certified trials' lifts
(EG_OPT_KICK_ROUNDS): whatever the slice length, the credits equal the
oracle's, and on road-like grids the jumps do raise vertices."""
from __future__ import annotations

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


GAMES = {
    "grid96": lambda: gen.grid_game(96, 96, seed=3),
    "grid200": lambda: gen.grid_game(200, 200, seed=5),
    "grid64x150": lambda: gen.grid_game(64, 150, seed=7),
    "varied": lambda: gen.varied_game(4000, 2, 5, 2000, seed=9),
    "uniform": lambda: gen.uniform_game(3000, 3, -40, 30, seed=11),
}


@pytest.mark.parametrize("kick", [0, 1, 2, 8])
@pytest.mark.parametrize("name", list(GAMES))
def test_cycle_jumps_keep_the_oracle_credits(name, kick):
    a = GAMES[name]()
    want = exact(a)
    with eg.Arena(a) as ar:
        ar.tune(kick_rounds=kick, certify_after=0)  # straight into the trials
        for bits in (0, 64):
            out, st = ar.solve(credit_bits=bits)
            assert st.status == eg.EG_OK
            np.testing.assert_array_equal(out, want)
            if kick == 0:
                assert st.cycle_jumps == 0


def test_cycle_jumps_raise_vertices_on_grids():
    a = gen.grid_game(256, 256, seed=2)
    want = exact(a)
    with eg.Arena(a) as ar:
        ar.tune(kick_rounds=1, certify_after=0)
        out, st = ar.solve(64)
        np.testing.assert_array_equal(out, want)
        assert st.cycle_jumps > 0
        ar.tune(kick_rounds=0)
        out0, st0 = ar.solve(64)
        np.testing.assert_array_equal(out0, want)
        assert st.rounds < st0.rounds


@pytest.mark.parametrize("k", [-50, 0, 60])
def test_cycle_jumps_under_threshold_views_and_int32(k):
    a = gen.grid_game(80, 80, seed=4)
    w2 = gen.threshold_weights(a.w, k, 10, scale=4)
    want = exact(a, w2)
    with eg.Arena(a) as ar:
        ar.tune(kick_rounds=1)
        for bits in (0, 64):
            out, _ = ar.solve(credit_bits=bits, w_scale=4, w_shift=k * 10)
            np.testing.assert_array_equal(out, want)
