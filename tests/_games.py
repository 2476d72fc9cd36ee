"""Test helpers: golden-file parsing, small arena builders, and closed forms
of the energy objective (Eq. 1, Sec. 3) for single-successor arenas."""
from __future__ import annotations

import os

import numpy as np

from paper_1710_03647_gb300.gen import Arena, pack_owner

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOP64 = np.iinfo(np.int64).max


def arena_from_edges(owners, edges, name="") -> Arena:
    """Edges (src, dst, w) kept in their given order inside each row."""
    n = len(owners)
    edges = sorted(enumerate(edges), key=lambda t: (t[1][0], t[0]))
    src = np.array([e[1][0] for e in edges], dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    col = np.array([e[1][1] for e in edges], dtype=np.int32)
    w = np.array([e[1][2] for e in edges], dtype=np.int32)
    return Arena(n, row_ptr, col, w, pack_owner(np.array(owners, dtype=bool)), name)


def load_hand_games(path=None):
    """Parse tests/golden/hand_games.txt into (arena, bound, expected) triples."""
    path = path or os.path.join(GOLDEN, "hand_games.txt")
    games, cur = [], None
    with open(path) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "game":
                cur = dict(name=tok[1], owners=None, edges=[], bound=None, expect=None)
            elif tok[0] == "owners":
                cur["owners"] = [int(x) for x in tok[1:]]
            elif tok[0] == "edge":
                cur["edges"].append((int(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "bound":
                cur["bound"] = int(tok[1])
            elif tok[0] == "expect":
                cur["expect"] = np.array([TOP64 if x == "T" else int(x) for x in tok[1:]], dtype=np.int64)
            elif tok[0] == "end":
                games.append((arena_from_edges(cur["owners"], cur["edges"], cur["name"]), cur["bound"],
                              cur["expect"]))
                cur = None
            else:
                raise ValueError(f"bad golden line: {raw!r}")
    return games


def functional_credit(succ, weight):
    """Minimum credits for an arena where every vertex has one successor.

    The play from v is fixed, so Eq. 1 asks for the least c >= 0 with
    c + (every prefix sum) >= 0.  The play enters a cycle; if its weight is
    negative the prefix sums are unbounded below (TOP), otherwise the lowest
    prefix sum is reached within the path to the cycle plus one lap.
    Computed by walking the play directly, with no lifting involved.
    """
    n = len(succ)
    out = np.zeros(n, dtype=np.int64)
    for v in range(n):
        seen = {}
        u, s, low, step = v, 0, 0, 0
        while u not in seen:
            seen[u] = (step, s)
            s += int(weight[u])
            low = min(low, s)
            u = int(succ[u])
            step += 1
        _, s_at_entry = seen[u]
        lap = s - s_at_entry
        if lap < 0:
            out[v] = TOP64
            continue
        # one more lap covers every prefix inside the cycle
        start = u
        while True:
            s += int(weight[u])
            low = min(low, s)
            u = int(succ[u])
            if u == start:
                break
        out[v] = -low
    return out
