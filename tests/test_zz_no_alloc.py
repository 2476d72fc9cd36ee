"""The allocation-free entry point, eg_solve_credit_noalloc.

It serves callers that cannot allocate device memory at solve time (a
framework that has reserved the GPU for its own allocator, or a latency-bound
loop that cannot afford the device-wide synchronisation of cudaMalloc and
cudaFree).  Here it must give exactly the credits of eg_solve_credit on the
same arena, on two calls in a row (the second reuses the library's working
array left over from the first), and refuse what it cannot hold.

This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1710_03647_gb300 import eg, gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


CASES = [
    ("uniform1k", lambda: gen.config(1, 1), 32, 1, 0),
    ("rmat14", lambda: gen.rmat_game(14, 8, seed=2), 32, 1, 0),
    ("grid64", lambda: gen.grid_game(64, 64, seed=1), 64, 1, 0),
    ("varied5k", lambda: gen.varied_game(5000, 2, 16, 1000, seed=3), 64, 1, 0),
    ("rmat12_threshold", lambda: gen.rmat_game(12, 8, seed=4), 64, 256, 9 * 100),
]


@pytest.mark.parametrize("name,make,bits,scale,shift", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_solve_twice(name, make, bits, scale, shift):
    a = make()
    dt = torch.int32 if bits == 32 else torch.int64
    with eg.Arena(a) as ar:
        want = torch.empty(a.n, dtype=dt, device="cuda:0")
        eg.eg_solve_credit(ar.handle, bits, scale, shift, want)
        for call in range(2):
            got = torch.full((a.n,), -7, dtype=dt, device="cuda:0")
            rc, st = eg.eg_solve_credit_noalloc(ar.handle, bits, scale, shift, got)
            torch.cuda.synchronize()
            assert rc == eg.EG_OK and st.credit_bits == bits
            np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy(), err_msg=f"call {call}")


def test_noalloc_refuses_what_it_cannot_hold():
    a = gen.uniform_game(eg.EG_NOALLOC_MAX_VERTICES + 1, 2, -3, 3, seed=5)
    with eg.Arena(a) as ar:
        out = torch.empty(a.n, dtype=torch.int64, device="cuda:0")
        with pytest.raises(eg.EGError) as ei:
            eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, out)
        assert ei.value.status == eg.EG_ERR_INVALID
        assert "at most" in str(ei.value)
    small = gen.config(1, 2)
    with eg.Arena(small) as ar:
        host = np.empty(small.n, dtype=np.int64)
        with pytest.raises(eg.EGError) as ei:  # the output must be device memory
            eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, host.ctypes.data)
        assert ei.value.status == eg.EG_ERR_INVALID
        dev = torch.empty(small.n, dtype=torch.int64, device="cuda:0")
        with pytest.raises(eg.EGError) as ei:  # no widening buffer: 32 or 64 only
            eg.eg_solve_credit_noalloc(ar.handle, 0, 1, 0, dev)
        assert ei.value.status == eg.EG_ERR_INVALID


def _certified_oracle(a):
    import oracle

    return oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)[0]


def test_noalloc_takes_the_certified_route_on_a_grid():
    # a 512 x 512 road-like grid: the plain cap-C lifting would climb for
    # hours; the allocation-free solve takes the same certified trials as
    # eg_solve_credit and reaches the same credits
    a = gen.grid_game(512, 512, seed=2)
    with eg.Arena(a) as ar:
        want = torch.empty(a.n, dtype=torch.int64, device="cuda:0")
        _, st_a = eg.eg_solve_credit(ar.handle, 64, 1, 0, want)
        for call in range(2):
            got = torch.full((a.n,), -7, dtype=torch.int64, device="cuda:0")
            rc, st = eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, got, max_rounds=200000)
            assert rc == eg.EG_OK and st.status == eg.EG_OK
            assert st.trials >= 1 and st.phases >= 3
            np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy(), err_msg=f"call {call}")
        np.testing.assert_array_equal(want.cpu().numpy(), _certified_oracle(a))


def test_noalloc_budget_leaves_credits_below_the_fixpoint():
    a = gen.grid_game(256, 256, seed=1)
    with eg.Arena(a) as ar:
        want = torch.empty(a.n, dtype=torch.int64, device="cuda:0")
        eg.eg_solve_credit(ar.handle, 64, 1, 0, want)
        ref = want.cpu().numpy()
        for rounds in (1, 12):
            got = torch.full((a.n,), -7, dtype=torch.int64, device="cuda:0")
            rc, st = eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, got, max_rounds=rounds, raise_on_error=False)
            assert st.status == rc
            g = got.cpu().numpy()
            if rounds == 1 or rc != eg.EG_OK:  # one round cannot reach the fixpoint of this grid
                assert rc == eg.EG_ERR_BUDGET
                assert (g >= 0).all() and (g <= ref).all()
            else:
                np.testing.assert_array_equal(g, ref)
        got = torch.empty(a.n, dtype=torch.int64, device="cuda:0")
        rc, st = eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, got)
        assert rc == eg.EG_OK
        np.testing.assert_array_equal(got.cpu().numpy(), ref)


def test_noalloc_refuses_misaligned_output():
    small = gen.config(1, 3)
    with eg.Arena(small) as ar:
        buf = torch.empty(small.n + 1, dtype=torch.int64, device="cuda:0")
        with pytest.raises(eg.EGError) as ei:  # 4 bytes off an 8-byte boundary
            eg.eg_solve_credit_noalloc(ar.handle, 64, 1, 0, buf.data_ptr() + 4)
        assert ei.value.status == eg.EG_ERR_INVALID and "aligned" in str(ei.value)


@pytest.mark.parametrize("sweeps,chunk", [(2, 32), (1, 1024)])
def test_noalloc_with_sweeps_and_chunks(sweeps, chunk):
    # the dense sweeps and chunked lists run in the allocation-free array too
    # (the sweeps use only the credits and round 0's push list); the credits
    # equal the allocating solve's and, on the grid, the oracle's
    for make, bits in ((lambda: gen.grid_game(96, 128, seed=6), 64), (lambda: gen.rmat_game(13, 8, seed=7), 32)):
        a = make()
        dt = torch.int32 if bits == 32 else torch.int64
        with eg.Arena(a) as ar:
            ar.tune(sweeps=sweeps, chunk_edges=chunk, certify_after=0)
            want = torch.empty(a.n, dtype=dt, device="cuda:0")
            eg.eg_solve_credit(ar.handle, bits, 1, 0, want)
            got = torch.full((a.n,), -7, dtype=dt, device="cuda:0")
            rc, st = eg.eg_solve_credit_noalloc(ar.handle, bits, 1, 0, got, max_rounds=200000)
            torch.cuda.synchronize()
            assert rc == eg.EG_OK and st.status == eg.EG_OK
            np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())
            if bits == 64:
                np.testing.assert_array_equal(want.cpu().numpy(), _certified_oracle(a))
