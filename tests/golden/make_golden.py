"""Writes the stored expected results of the full-size parity tests.

Calls only the CPU oracle (Algorithm 1 of arXiv 1710.03647, Sec. 3.1) and the
seeded input generators; never the CUDA path.  For each workload it stores the
SHA-256 of the oracle's int64 credit array (TOP = INT64_MAX) together with a few
summary figures, in tests/golden/<name>.json.

    python tests/golden/make_golden.py rmat20_s1
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

WORKLOADS = {
    # R-MAT scale 20, edge factor 8, weights in [-100, 100], seed 1
    "rmat20_s1": lambda: gen.config(2, seed=1),
    "rmat18_s1": lambda: gen.rmat_game(18, 8, seed=1),
}


def credit_digest(f: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(f, dtype=np.int64).tobytes()).hexdigest()


def main(name: str) -> None:
    a = WORKLOADS[name]()
    t0 = time.time()
    f, st = oracle.solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
    dt = time.time() - t0
    top = f == oracle.TOP
    rec = dict(workload=name, n=a.n, m=a.m, C=st["C"], sha256=credit_digest(f), top=int(top.sum()),
               finite_sum=int(f[~top].sum()), finite_max=int(f[~top].max()) if (~top).any() else -1,
               oracle_lifts=st["lifts"], oracle_lift_edge_evals=st["lift_edge_evals"],
               oracle_pre_scans=st["pre_scans"], oracle_seconds=round(dt, 1))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        main(nm)
