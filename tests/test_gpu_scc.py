"""GPU tests of SCC-ordered solving (EG_OPT_SCC_ORDER, eg_scc_info,
eg_scc_levels): the device condensation has the components scipy finds and
levels that order them topologically, and solving level by level gives the
oracle's credits, with and without the warm start."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1710_03647_gb300 import eg, gen

pytestmark = pytest.mark.gpu
scipy_graph = pytest.importorskip("scipy.sparse.csgraph")
sparse = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__

    __graft_entry__.build()
    eg.load()


def exact(a, w=None):
    f, _ = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w if w is None else w, a.owner_bits)
    return f


def packed(games):
    from paper_1710_03647_gb300.gen import Arena

    n, row_ptr, col, w, owner_bits, _ = eg.pack_games(games)
    return Arena(n, row_ptr, col, w, owner_bits, "packed")


def chain_of_cycles(k=40, seed=3):
    """k small cycles, each with an edge to the next: k components in k levels."""
    s = gen.Stream(seed, 21)
    edges = []
    for c in range(k):
        a, b = 2 * c, 2 * c + 1
        edges += [(a, b), (b, a)]
        if c + 1 < k:
            edges.append((b, 2 * c + 2))
    src = np.array([e[0] for e in edges])
    dst = np.array([e[1] for e in edges])
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    n = 2 * k
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    w = s.integers(len(dst), -6, 6).astype(np.int32)
    owner = gen.pack_owner(gen.Stream(seed, 22).unit(n) < 0.5)
    return gen.Arena(n, row_ptr, dst.astype(np.int32), w, owner, "chain")


GAMES = {
    "rmat14": lambda: gen.rmat_game(14, 8, seed=2),
    "rmat12_sparse": lambda: gen.rmat_game(12, 2, seed=5),
    "mixed_batch": lambda: packed([gen.config(1, 2), gen.varied_game(1500, 2, 6, 50, seed=3),
                                   gen.rmat_game(10, 4, seed=4), gen.grid_game(20, 24, seed=2),
                                   gen.tiny_game(30, 3, -4, 4, seed=5)]),
    "chain": chain_of_cycles,
    "grid48": lambda: gen.grid_game(48, 48, seed=1),
}


@pytest.mark.parametrize("name", list(GAMES))
def test_condensation_matches_scipy_and_orders_levels(name):
    a = GAMES[name]()
    with eg.Arena(a) as ar:
        info = eg.eg_scc_info(ar.handle)
        level, comp = eg.eg_scc_levels(ar.handle, a.n)
    src = np.repeat(np.arange(a.n), np.diff(np.asarray(a.row_ptr)))
    g = sparse.csr_matrix((np.ones(a.m), (src, np.asarray(a.col))), shape=(a.n, a.n))
    ncomp, labels = scipy_graph.connected_components(g, directed=True, connection="strong")
    assert info["components"] == ncomp
    # same partition: the map label -> comp is a bijection
    pairs = set(zip(labels.tolist(), comp.tolist()))
    assert len(pairs) == ncomp
    # each component is named by its largest vertex id
    for lab in np.unique(labels)[:200]:
        members = np.nonzero(labels == lab)[0]
        assert (comp[members] == members.max()).all()
    # levels: an edge never climbs, and leaves its component only downwards;
    # a component's level is one more than the highest it reaches (0 if none)
    dst = np.asarray(a.col)
    assert (level[src] >= level[dst]).all()
    cross = comp[src] != comp[dst]
    assert (level[src][cross] > level[dst][cross]).all()
    best = np.full(a.n, -1, dtype=np.int64)
    np.maximum.at(best, comp[src][cross], level[dst][cross])
    roots = np.unique(comp)
    assert (level[roots] == best[roots] + 1).all()
    assert info["levels"] == level.max() + 1


@pytest.mark.parametrize("warm", [1, 0])
@pytest.mark.parametrize("name", ["rmat14", "mixed_batch", "chain", "grid48"])
def test_scc_ordered_solve_equals_oracle(name, warm):
    a = GAMES[name]()
    want = exact(a)
    with eg.Arena(a) as ar:
        levels = eg.eg_scc_info(ar.handle)["levels"]
        ar.tune(scc_order=1, warm_start=warm)
        for bits in (0, 64):
            out, st = ar.solve(credit_bits=bits)
            assert st.status == eg.EG_OK
            np.testing.assert_array_equal(out, want)
            kinds = {p["kind"] for p in st.phase_list()}
            # one level (a grid) orders nothing and takes the default route
            assert (kinds == {"level"}) == (levels > 1), (levels, kinds)
        # the threshold view too
        w2 = gen.threshold_weights(a.w, 17, 3)
        out, _ = ar.solve(credit_bits=64, w_scale=256, w_shift=17 * 3)
        np.testing.assert_array_equal(out, exact(a, w2))


def test_scc_ordered_budget_stays_below_the_fixpoint():
    a = chain_of_cycles(60, seed=8)
    want = exact(a)
    with eg.Arena(a) as ar:
        ar.tune(scc_order=1)
        out = np.empty(a.n, dtype=np.int64)
        rc, st = eg.eg_solve_credit(ar.handle, 64, 1, 0, out, max_rounds=1, raise_on_error=False)
        if rc != eg.EG_OK:
            assert rc == eg.EG_ERR_BUDGET
        assert (out <= want).all() and (out >= 0).all()
        out, _ = ar.solve(64)
        np.testing.assert_array_equal(out, want)


def test_single_level_condensation_takes_the_default_route():
    # a grid is one component: the SCC-ordered route would be the plain
    # lifting with cap C, so the solve takes the certified route instead
    a = gen.grid_game(128, 128, seed=6)
    with eg.Arena(a) as ar:
        assert eg.eg_scc_info(ar.handle)["levels"] == 1
        ar.tune(scc_order=1)
        out, st = ar.solve(64)
        assert "level" not in {p["kind"] for p in st.phase_list()}
        np.testing.assert_array_equal(out, exact(a))
