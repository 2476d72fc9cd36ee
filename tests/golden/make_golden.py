"""Writes the stored expected results of the full-size parity tests.

Calls only the CPU oracle (Algorithm 1 of arXiv 1710.03647, Sec. 3.1, and
`oracle.certified_solve`, which composes capped Algorithm 1 runs) and the
seeded input generators; never the CUDA path.  For each workload it stores
the SHA-256 of the oracle's int64 credit array (TOP = INT64_MAX) together with
a few summary figures, in tests/golden/<name>.json.

    python tests/golden/make_golden.py rmat20_s1 grid4000_s1 batch4096_sample thresholds_rmat20

  rmat20_s1, rmat18_s1  Algorithm 1 with cap C = M_G, as the paper runs it
  grid4000_s1           the 4000 x 4000 road-like grid (16M vertices); a
                        cap-C run would need ~1e14 lifts, so the certified
                        composition decides it with small caps
  batch4096_sample      32 games of the 4096-game batch, spread over its
                        size range (every 128th game in order of n)
  thresholds_rmat20     three threshold queries w' = 256 w - k * 100,
                        k in {-128, 0, 127}, on the R-MAT scale-20 arena
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_03647_gb300 import gen  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
BATCH_COUNT = 4096
BATCH_SAMPLES = 32
THRESHOLD_KS = (-128, 0, 127)
THRESHOLD_W = 100


def credit_digest(f: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(f, dtype=np.int64).tobytes()).hexdigest()


def summary(f: np.ndarray) -> dict:
    top = f == oracle.TOP
    return dict(sha256=credit_digest(f), top=int(top.sum()), finite_sum=int(f[~top].sum()),
                finite_max=int(f[~top].max()) if (~top).any() else -1)


def plain(a) -> dict:
    t0 = time.time()
    f, st = oracle.solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
    dt = time.time() - t0
    return dict(n=a.n, m=a.m, C=st["C"], **summary(f), oracle_lifts=st["lifts"],
                oracle_lift_edge_evals=st["lift_edge_evals"], oracle_pre_scans=st["pre_scans"],
                oracle_seconds=round(dt, 1))


def certified(a, w=None) -> dict:
    w = a.w if w is None else w
    t0 = time.time()
    f, st = oracle.certified_solve(a.n, a.row_ptr, a.col, w, a.owner_bits,
                                   log=lambda s: print(f"  {a.name}: {s}", flush=True))
    dt = time.time() - t0
    return dict(n=a.n, m=a.m, C=st["C"], **summary(f), route="certified", trial=st["trial"], B=st["B"],
                K=st["K"], oracle_lifts=st["lifts"], oracle_lift_edge_evals=st["lift_edge_evals"],
                oracle_pre_scans=st["pre_scans"], oracle_seconds=round(dt, 1))


def batch_sample_indices(shapes) -> list[int]:
    """Every (count / samples)-th game in order of size, smallest to largest."""
    order = sorted(range(len(shapes)), key=lambda i: (shapes[i][0], i))
    step = len(order) // BATCH_SAMPLES
    return [order[step // 2 + j * step] for j in range(BATCH_SAMPLES)]


def batch4096_sample() -> dict:
    shapes = gen.batch_shapes(BATCH_COUNT)
    games = []
    for i in batch_sample_indices(shapes):
        n, W = shapes[i]
        a = gen.batch_game(i, n, W)
        games.append(dict(index=i, W=W, **certified(a)))
        print(json.dumps(games[-1]), flush=True)
    return dict(count=BATCH_COUNT, games=games)


def thresholds_rmat20() -> dict:
    a = gen.config(2, seed=1)
    out = []
    for k in THRESHOLD_KS:
        w2 = gen.threshold_weights(a.w, k, THRESHOLD_W)
        out.append(dict(k=k, scale=256, shift=k * THRESHOLD_W, **certified(a, w2)))
        print(json.dumps(out[-1]), flush=True)
    return dict(W=THRESHOLD_W, queries=out)


WORKLOADS = {
    # R-MAT scale 20, edge factor 8, weights in [-100, 100], seed 1
    "rmat20_s1": lambda: plain(gen.config(2, seed=1)),
    "rmat18_s1": lambda: plain(gen.rmat_game(18, 8, seed=1)),
    "grid4000_s1": lambda: certified(gen.config(3, seed=1)),
    "batch4096_sample": batch4096_sample,
    "thresholds_rmat20": thresholds_rmat20,
}


def main(name: str) -> None:
    rec = dict(workload=name, **WORKLOADS[name]())
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec)[:2000])


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        main(nm)
