"""Command-line solve of a generated workload through the C ABI.

    python -m paper_1710_03647_gb300.cli --workload grid --side 2000 --bits 64 \
        --local-windows 0 --max-rounds 30 --repeat 3
    python -m paper_1710_03647_gb300.cli --workload batch --games 128 --repeat 3

Builds the arena with the seeded generators of `gen`, applies the given
solver options and prints the counters of every solve as one JSON line.  A
round budget that runs out is reported, not raised (status -7).  The batch
workload packs the first G games of the uneven batch (n log-uniform in
[1k, 200k], out-degree uniform in [2, 16], W log-uniform in [10, 10^4]) into
one arena and solves them all in one plan (one persistent launch).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from paper_1710_03647_gb300 import eg, gen


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=["uniform", "rmat", "grid", "varied", "batch"], default="rmat")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale (2^scale vertices)")
    ap.add_argument("--side", type=int, default=4000, help="grid side")
    ap.add_argument("--n", type=int, default=100000, help="vertices of uniform / varied games")
    ap.add_argument("--games", type=int, default=128, help="games of the batch workload")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--bits", type=int, default=0, choices=[0, 32, 64])
    ap.add_argument("--max-rounds", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    for opt in ("local-windows", "local-maxdeg", "warm-start", "cap-certify", "certify-after", "dual-k",
                "blocks-per-sm", "scc-order", "kick-rounds", "sweeps", "chunk-edges"):
        ap.add_argument("--" + opt, type=int, default=None)
    args = ap.parse_args(argv)
    if args.workload == "batch":
        batch(args)
        return
    if args.workload == "rmat":
        a = gen.rmat_game(args.scale, 8, seed=args.seed)
    elif args.workload == "grid":
        a = gen.grid_game(args.side, args.side, seed=args.seed)
    elif args.workload == "uniform":
        a = gen.uniform_game(args.n, 4, -10, 10, seed=args.seed)
    else:
        a = gen.varied_game(args.n, 2, 16, 1000, seed=args.seed)
    with eg.Arena(a) as arena:
        arena.tune(local_windows=args.local_windows, local_maxdeg=args.local_maxdeg, warm_start=args.warm_start,
                   cap_certify=args.cap_certify, certify_after=args.certify_after, dual_k=args.dual_k,
                   blocks_per_sm=args.blocks_per_sm, scc_order=args.scc_order, kick_rounds=args.kick_rounds,
                   sweeps=args.sweeps, chunk_edges=args.chunk_edges)
        out = np.empty(a.n, dtype=np.int32 if args.bits == 32 else np.int64)
        for _ in range(args.repeat):
            rc, st = eg.eg_solve_credit(arena.handle, args.bits, 1, 0, out, max_rounds=args.max_rounds,
                                        raise_on_error=False)
            print(json.dumps({"workload": args.workload, "n": a.n, "m": a.m, "status": rc, **st.as_dict()}),
                  flush=True)


def batch(args) -> None:
    games = gen.batch_games(args.games, seed=args.seed)
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(games)
    with eg.Arena(gen.Arena(n, row_ptr, col, w, owner_bits, "batch")) as arena:
        arena.tune(local_windows=args.local_windows, local_maxdeg=args.local_maxdeg, warm_start=args.warm_start,
                   cap_certify=args.cap_certify, certify_after=args.certify_after, dual_k=args.dual_k,
                   blocks_per_sm=args.blocks_per_sm, kick_rounds=args.kick_rounds, sweeps=args.sweeps,
                   chunk_edges=args.chunk_edges)
        eg.eg_set_parts(arena.handle, part_ptr)
        with eg.Plan(arena.handle, args.games, credit_bits=args.bits) as plan:
            for _ in range(args.repeat):
                _, st = plan.run(max_rounds=args.max_rounds, raise_on_error=False)
                print(json.dumps({"workload": "batch", "games": args.games, "n": int(n), "m": int(row_ptr[-1]),
                                  **st.as_dict()}), flush=True)


if __name__ == "__main__":
    main()
