"""GPU tests of the certified trials' credit widths.  A trial lift whose cap
plus largest weight fits int32 runs in int32 state, whatever the width of the
solve; the others run in int64; an exact capped fixpoint computed in int32 is
widened into the solve's own state.  The trial caps scale with max|w'|
(B = 4 max|w'| 4^k, dual cap (K + 1) B), so scaling the weights of a road-like
grid moves the trials across the int32 limit:

  scale 1, 1000   every lift in int32 (the solve itself in int32 or int64)
  scale 1e5       the capped lifts in int32, the dual lifts in int64
  scale 1e6       every lift in int64

In every case the credits equal the oracle's certified composition of
capped Algorithm 1 runs (Sec. 3.1) on the scaled weights, element by element.
"""
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


@pytest.mark.parametrize("scale", [1, 1000, 100000, 1000000])
def test_trial_widths_keep_the_oracle_credits(scale):
    a = gen.grid_game(100, 100, seed=12)
    w2 = np.asarray(a.w, dtype=np.int64) * scale
    want, ost = oracle.certified_solve(a.n, a.row_ptr, a.col, w2, a.owner_bits)
    with eg.Arena(a) as ar:
        ar.tune(certify_after=0)  # straight into the trials
        for bits in (0, 64):
            out, st = ar.solve(credit_bits=bits, w_scale=scale)
            assert st.status == eg.EG_OK and st.C == ost["C"]
            assert st.trials >= 1
            np.testing.assert_array_equal(out, want, err_msg=f"bits={bits}")


def test_trial_widths_into_a_device_buffer():
    import torch

    a = gen.grid_game(64, 96, seed=13)
    want, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
    with eg.Arena(a) as ar:
        ar.tune(certify_after=0, sweeps=1)
        out = torch.full((a.n,), -1, dtype=torch.int64, device="cuda")
        _, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out)
        assert st.status == eg.EG_OK and st.credit_bits == 64
        np.testing.assert_array_equal(out.cpu().numpy(), want)
