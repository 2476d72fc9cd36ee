#!/usr/bin/env python3
"""Benchmark: least-fixpoint lifting of the energy progress measure on the
4000 x 4000 road-like grid game (16M vertices, 64.6M edges, weights in
[-1000, 1000] with 40% negative, int64 credits), solved to the exact fixpoint
per step by eg_solve_credit's default route (a short cap-C attempt, then
certified trial caps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Metric: edge-relaxations/s, i.e. evaluations
of f(u) (-) w over edges (pulls of player-0 lifts plus pushes to
predecessors) divided by the device time of the solve; time-to-fixpoint per
step is ms_per_step, shown beside the CPU oracle's time on the same game.
The arena is resident in HBM before the timed region; between timed steps a
512 MiB buffer is rewritten to flush L2 (the arena and state, ~3.5 GB, are
larger than L2 anyway).

--impl reference times the CPU oracle on a bounded sample of the same
workload: the same generator at 700 x 700 per step, solved exactly by the
oracle's certified composition of Algorithm 1 runs.

A single game does not shard: with --gpus N every rank solves its own
replica (no collective on the data path) and value sums the ranks' work
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="grid4000_s1: 4000x4000 grid, 4-neighbour directed edges + 1% uniform long edges, "
                         "w negative w.p. 0.4 (uniform in [-1000,-1]) else uniform in [0,1000], "
                         "owner Bernoulli(0.5), seed 1",
                side=4000, seed=1, credit_bits=64, golden="grid4000_s1")
CONTEXT_RMAT = dict(workload="rmat20_s1: R-MAT scale 20 (a,b,c,d)=(.57,.19,.19,.05), 8*2^20 draws, "
                             "w uniform in [-100,100], owner Bernoulli(0.5), seed 1",
                    scale=20, seed=1, credit_bits=32, golden="rmat20_s1")
SAMPLE_SIDE = 700      # the reference arm's per-step sample of the headline workload
BASELINE_SIDE = 1000   # cpu_baseline's sample (one solve, ~6-10 s)
METRIC = "edge-relaxations/s"
UNIT = "relax/s"


# algorithmic bytes (per unit): relaxation = index 4 + weight 4 + credit s;
# list entry (lift or push) = two offsets 8 + entry 4 + credit s;
# enqueue = entry write 4 + bitmap word 4
def algorithmic_bytes(st, s):
    return st["relaxations"] * (8 + s) + (st["lifts"] + st["pushes"]) * (12 + s) + st["enqueues"] * 8


INT32_ROOM = 2**31 - 2  # largest cap + |weight| an int32 credit array holds below its TOP


def lift_widths(st, wmax):
    """Credit width (bits) of each lifting launch of a single-game solve, by
    the library's rule: a trial lift (capped, or the dual with weights
    -(K w' + 1)) whose cap plus largest |weight| fits int32 computes in
    int32; the other launches at the solve's width.  K of a dual is its cap
    over the preceding capped lift's cap, minus one."""
    out, B = [], None
    for p in st["phase_list"]:
        if p["kind"] == "capped":
            B = p["cap"]
            out.append(32 if B + wmax <= INT32_ROOM else st["credit_bits"])
        elif p["kind"] == "dual" and B:
            K = p["cap"] // B - 1
            out.append(32 if p["cap"] + K * wmax + 1 <= INT32_ROOM else 64)
        else:
            out.append(st["credit_bits"])
    return out


def credit_bytes(st, wmax):
    """Bytes per credit of a solve's lifting, its launches weighted by their
    relaxations (the trial lifts may compute narrower than the solve)."""
    w = lift_widths(st, wmax)
    rel = [p["relaxations"] for p in st["phase_list"]]
    if not w or sum(rel) == 0:
        return st["credit_bits"] / 8
    return sum(r * b for r, b in zip(rel, w)) / sum(rel) / 8


def launches_of(st, sweeps=0):
    """Kernels of one single-game solve: warm start, init, `sweeps` dense
    sweeps and the fixpoint per fixpoint launch, plus the trials' bitmap
    passes (3 after a capped lift, 2 after a dual lift)."""
    kinds = [p["kind"] for p in st["phase_list"]]
    return (3 + sweeps) * len(kinds) + 3 * kinds.count("capped") + 2 * kinds.count("dual")


def strip_comments(src):
    """C/C++ source without // and /* */ comments (string and character
    literals kept), so that a comment edit does not count as a kernel change."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "".join(out)


def kernel_source_hash():
    """SHA-256 over the sources the fixpoint kernel is compiled from, comments
    stripped and whitespace runs collapsed."""
    import hashlib

    h = hashlib.sha256()
    for name in ("eg_solve.cu", "eg_device.cuh", "eg_internal.h"):
        with open(os.path.join(ROOT, "paper_1710_03647_gb300", "csrc", name)) as fh:
            h.update(" ".join(strip_comments(fh.read()).split()).encode())
    return h.hexdigest()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 20 ms from before
    the warm-up to the end of the timed region; each sample is stamped with
    the host time it arrived, and mark() brackets the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, begin):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        inside = [r for t, r in self.rows if self.t0 is not None and self.t0 <= t <= (self.t1 or t) + 0.03]
        window = "timed"
        rows = inside
        if not rows:
            rows, window = [r for _, r in self.rows], "warm-up and timed"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


def reduce_over_ranks(total_ms, relax, device, dist):
    """Replicas: the job's time is the slowest rank's, its work the sum."""
    import torch

    t = torch.tensor([float(total_ms), float(relax)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_work(st):
    """Edge evaluations of the oracle: lift edges, predecessor scans, recounts."""
    return st["lift_edge_evals"] + st["pre_scans"] + st["recount_evals"]


def run_reference(args, world, rank):
    """The CPU oracle (certified composition of Algorithm 1 runs, one
    thread) on a bounded sample of the headline workload per step."""
    if rank != 0:
        return
    import oracle
    from paper_1710_03647_gb300 import gen

    a = gen.grid_game(SAMPLE_SIDE, SAMPLE_SIDE, seed=WORKLOAD["seed"])
    times, relax = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, st = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            relax.append(oracle_work(st))
    value = sum(relax) / sum(times)
    sample = (f"oracle (certified composition of Algorithm 1 runs, 1 thread) on the {SAMPLE_SIDE}x{SAMPLE_SIDE} grid "
              f"(n={a.n}, m={a.m}) from the same generator and seed, one exact solve per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": WORKLOAD["workload"], "sample": f"{SAMPLE_SIDE}x{SAMPLE_SIDE}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline():
    """The oracle as it stands, single-threaded, on a bounded sample (~10 s)."""
    import oracle
    from paper_1710_03647_gb300 import gen

    a = gen.grid_game(BASELINE_SIDE, BASELINE_SIDE, seed=WORKLOAD["seed"])
    t0 = time.perf_counter()
    _, st = oracle.certified_solve(a.n, a.row_ptr, a.col, a.w, a.owner_bits)
    dt = time.perf_counter() - t0
    return {"value": oracle_work(st) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{BASELINE_SIDE}x{BASELINE_SIDE} grid (n={a.n}, m={a.m}) from the headline's generator, one "
                      f"exact solve by the oracle's certified composition of Algorithm 1 runs ({dt:.1f} s, "
                      f"{oracle_work(st)} edge evaluations)"}


def ev_pair():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    return json.load(open(path)) if os.path.exists(path) else None


def traffic_record(name, settings=None):
    """DRAM bytes per solve from the committed ncu record, or None when the
    kernel sources changed since it was taken or the record was taken with
    other launch settings than `settings` (the ones timed)."""
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    rec = json.load(open(prof))
    if rec.get("kernel_source_sha256") != kernel_source_hash():
        return None
    if settings is not None and any(rec.get("settings", {}).get(k) != v for k, v in settings.items()):
        return None
    return rec.get("dram_bytes_per_solve")


SETTING_KEYS = ("local_windows", "local_maxdeg", "blocks_per_sm", "cap_certify", "certify_after", "dual_k",
                "kick_rounds", "sweeps", "chunk_edges")
DEFAULT_SETTINGS = dict(local_windows=64, local_maxdeg=64, blocks_per_sm=0, cap_certify=4, certify_after=8, dual_k=4,
                        kick_rounds=2, sweeps=0, chunk_edges=1024)


def rmat_context(eg, gen, torch, dev, stream, flush, plain_start=True, tune=True, scc=True):
    """Config 2 (R-MAT scale 20, int32): time to the fixpoint, relaxations/s
    and the fixpoint kernel against HBM, beside the oracle's stored time on
    the same game; optionally the paper's f = 0 start."""
    a = gen.rmat_game(CONTEXT_RMAT["scale"], 8, seed=CONTEXT_RMAT["seed"])
    bits = CONTEXT_RMAT["credit_bits"]
    s = bits // 8
    arena = eg.Arena(a)
    out = torch.empty(a.n, dtype=torch.int32, device=dev)
    for _ in range(3):
        eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
    tuning = None
    if tune:
        import tempfile

        with tempfile.TemporaryDirectory() as td:
            tuning = eg.eg_autotune(arena.handle, bits, 1, 0, os.path.join(td, "plans.jsonl"), max_solves=80)
    res = []
    for k in range(10):
        with torch.cuda.stream(stream):
            flush.fill_(k)
        b, e = ev_pair()
        b.record(stream)
        _, st = eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
        e.record(stream)
        torch.cuda.synchronize()
        res.append((b.elapsed_time(e), st.as_dict()))
    ms = statistics.median(r[0] for r in res)
    relax = sum(r[1]["relaxations"] for r in res)
    fix_ms = sum(r[1]["fixpoint_ms"] for r in res)
    wmax = int(np.abs(np.asarray(a.w, dtype=np.int64)).max())
    bytes_alg = sum(algorithmic_bytes(r[1], credit_bytes(r[1], wmax)) for r in res)
    peak, peak_kind = peaks()
    g = golden(CONTEXT_RMAT["golden"])
    out_d = {"workload": CONTEXT_RMAT["workload"], "n": a.n, "m": a.m, "credit_bits": bits,
             "time_to_fixpoint_ms": ms, "relax_per_s": relax / (sum(r[0] for r in res) * 1e-3),
             "rounds": res[-1][1]["rounds"], "relaxations_per_solve": res[-1][1]["relaxations"],
             "roofline": {"bound": "hbm", "achieved": bytes_alg / (fix_ms * 1e-3) / 1e9, "peak": peak,
                          "unit": "GB/s", "frac": bytes_alg / (fix_ms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
                          "traffic": traffic_record("fixpoint_rmat20_traffic.json",
                                                    {k: tuning[k] for k in SETTING_KEYS} if tuning
                                                    else dict(DEFAULT_SETTINGS)),
                          "kernel": "k_sweep + k_fixpoint (the lifting kernels)"},
             "oracle": None, "settings": "autotuned (eg_autotune)" if tuning else "defaults", "tuning": tuning}
    if g:
        out_d["oracle"] = {"time_to_fixpoint_s": g["oracle_seconds"], "route": "Algorithm 1 with cap C, 1 thread",
                           "edge_evaluations": g["oracle_lift_edge_evals"] + g["oracle_pre_scans"],
                           "speedup": g["oracle_seconds"] * 1e3 / ms}
    if plain_start:
        arena.tune(warm_start=0)
        _, pst = eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
        arena.tune(warm_start=1)
        pd = pst.as_dict()
        out_d["plain"] = {"time_to_fixpoint_ms": pd["ms"], "relaxations": pd["relaxations"], "rounds": pd["rounds"],
                          "note": "same solver, warm start and certified trials off (f = 0 start as in the paper)"}
    if scc:
        # SCC-ordered solving (levels of the condensation in turn): the
        # default warm start, and the paper's f = 0 start
        t0 = time.perf_counter()
        info = eg.eg_scc_info(arena.handle)
        info["condensation_ms"] = (time.perf_counter() - t0) * 1e3
        arena.tune(scc_order=1)
        sms = []
        for _ in range(5):
            b, e = ev_pair()
            b.record(stream)
            _, sst = eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
            e.record(stream)
            torch.cuda.synchronize()
            sms.append(b.elapsed_time(e))
        info["warm_time_to_fixpoint_ms"] = statistics.median(sms)
        info["warm_relaxations"] = sst.relaxations
        if plain_start:
            arena.tune(warm_start=0)
            _, pst = eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
            arena.tune(warm_start=1)
            info["plain_time_to_fixpoint_ms"] = pst.ms
            info["plain_relaxations"] = pst.relaxations
            info["plain_rounds"] = pst.rounds
        arena.tune(scc_order=0)
        out_d["scc_ordered"] = info
    return arena, a, out_d


def batch_games(eg, gen, torch, dev, stream, count, tune=True):
    """`count` uneven games (n log-uniform in [1k, 200k], out-degree uniform
    in [2, 16], weights in [-W, W], W log-uniform in [10, 10^4]): all in one
    persistent launch (a plan over one packed arena) vs one solve per game."""
    games = gen.batch_games(count)
    n, row_ptr, col, w, owner_bits, part_ptr = eg.pack_games(games)
    h = eg.eg_create(n, int(row_ptr[-1]), row_ptr, col, w, owner_bits=owner_bits)
    eg.eg_set_parts(h, part_ptr)
    t0 = time.perf_counter()
    scc = eg.eg_scc_info(h)  # the condensation of all games: how much SCC ordering could order
    scc["condensation_ms"] = (time.perf_counter() - t0) * 1e3
    plan = eg.Plan(h, count)
    bout = torch.empty(plan.total, dtype=torch.int64, device=dev)
    plan.run(bout, stream=stream.cuda_stream)
    tuning = None
    if tune:
        import tempfile

        with tempfile.TemporaryDirectory() as td:
            tuning = eg.eg_plan_autotune(plan, os.path.join(td, "plans.jsonl"), max_solves=80)
    bms = []
    for _ in range(3):
        b, e = ev_pair()
        b.record(stream)
        _, bst = plan.run(bout, stream=stream.cuda_stream)
        e.record(stream)
        torch.cuda.synchronize()
        bms.append(b.elapsed_time(e))
    batched = bout.cpu().numpy()
    plan.close()
    eg.eg_destroy(h)
    # one solve (one persistent launch) per game, each game's arena resident
    arenas = [eg.Arena(g) for g in games]
    outs = [torch.empty(g.n, dtype=torch.int64, device=dev) for g in games]
    for ar, o in zip(arenas[:8], outs[:8]):
        eg.eg_solve_credit(ar.handle, 0, 1, 0, o, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    per = []
    t0, t1 = ev_pair()
    t0.record(stream)
    for ar, o in zip(arenas, outs):
        b, e = ev_pair()
        b.record(stream)
        eg.eg_solve_credit(ar.handle, 0, 1, 0, o, stream=stream.cuda_stream)
        e.record(stream)
        per.append((b, e))
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1)
    lat = sorted(b.elapsed_time(e) for b, e in per)
    same = all(np.array_equal(o.cpu().numpy(), batched[int(part_ptr[i]):int(part_ptr[i + 1])])
               for i, o in enumerate(outs))
    for ar in arenas:
        ar.close()
    bmed = statistics.median(bms)
    return {"games": count, "vertices": int(n), "edges": int(row_ptr[-1]),
            "batched_ms": bmed, "batched_games_per_s": count / (bmed * 1e-3), "batched_relaxations": bst.relaxations,
            "per_game_total_ms": total, "per_game_games_per_s": count / (total * 1e-3),
            "per_game_p50_ms": lat[len(lat) // 2], "per_game_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "batched_equals_per_game": bool(same), "plan_tuning": tuning, "condensation": scc,
            "note": "batched: one plan (one persistent launch, CUDA graph replay) over a packed arena, tuned by "
                    "eg_plan_autotune; latency of every game in the batch = the batch time; per game: one "
                    "eg_solve_credit per resident arena with the library defaults"}


def _rmat_game(args):
    from paper_1710_03647_gb300 import gen

    scale, seed = args
    return gen.rmat_game(scale, 8, seed=seed)


def serving(eg, gen, torch, dev, stream, per_rate, scales=(10, 21), seed=11):
    """Poisson arrivals of R-MAT games (scale uniform in [lo, hi], so n is
    log-uniform in [2^lo, 2^hi]; weights in [-100, 100]) served by the
    continuous-batching server vs. one solve at a time in arrival order, at
    rates 0.25x-4x the serial capacity."""
    import multiprocessing as mp
    import threading

    rng = np.random.default_rng(seed)
    jobs = [(int(sc), 100 + i) for i, sc in enumerate(range(scales[0], scales[1] + 1))]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as workers:
        pool = workers.map(_rmat_game, jobs, chunksize=1)
    arenas = [eg.Arena(g) for g in pool]
    # credits land in pinned host memory on both routes, as the server's do
    out = torch.empty(max(g.n for g in pool), dtype=torch.int64, pin_memory=True)
    # serial capacity: solves back to back
    order = rng.integers(len(pool), size=per_rate)
    for k in range(len(pool)):
        eg.eg_solve_credit(arenas[k].handle, 0, 1, 0, out, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in order:
        eg.eg_solve_credit(arenas[k].handle, 0, 1, 0, out, stream=stream.cuda_stream)
    cap = per_rate / (time.perf_counter() - t0)
    rows = []
    for mult in (0.25, 0.5, 1.0, 2.0, 4.0):
        rate = mult * cap
        gaps = rng.exponential(1.0 / rate, size=per_rate)
        arrive = np.cumsum(gaps)
        picks = rng.integers(len(pool), size=per_rate)
        # serial: one solve at a time, in arrival order
        lat_s = []
        start = time.perf_counter()
        for t_arr, k in zip(arrive, picks):
            now = time.perf_counter() - start
            if now < t_arr:
                time.sleep(t_arr - now)
            eg.eg_solve_credit(arenas[k].handle, 0, 1, 0, out, stream=stream.cuda_stream)
            lat_s.append(time.perf_counter() - start - t_arr)
        span_s = time.perf_counter() - start
        # server: a submitting thread at the arrival times, polling here; one
        # untimed pass over the game pool first, so that the server's pinned
        # result buffers exist (as in a server that has been running)
        server = eg.eg_server_create(16 << 30, 64)
        for k in range(len(pool)):
            t = eg.eg_submit(server, arenas[k].handle, 0, 1, 0)
            while eg.eg_poll(server, t)[0] == eg.EG_PENDING:
                time.sleep(0.0002)
        tickets = [None] * per_rate
        start = time.perf_counter()

        def submit():
            for i, (t_arr, k) in enumerate(zip(arrive, picks)):
                now = time.perf_counter() - start
                if now < t_arr:
                    time.sleep(t_arr - now)
                tickets[i] = eg.eg_submit(server, arenas[k].handle, 0, 1, 0)

        th = threading.Thread(target=submit)
        th.start()
        lat_v, pending, done_at = [], set(range(per_rate)), 0.0
        while pending:
            for i in list(pending):
                if tickets[i] is None:
                    continue
                rc, st = eg.eg_poll(server, tickets[i])
                if rc == eg.EG_PENDING:
                    continue
                if rc != eg.EG_OK:
                    raise RuntimeError(f"served request failed: {rc} {eg.eg_last_error()}")
                lat_v.append(st.ms * 1e-3)
                pending.discard(i)
                done_at = time.perf_counter() - start
            time.sleep(0.0002)
        th.join()
        eg.eg_server_destroy(server)

        def pct(v, q):
            v = sorted(v)
            return 1e3 * v[min(len(v) - 1, int(q * len(v)))]

        rows.append({"rate_x_serial_capacity": mult, "offered_games_per_s": rate,
                     "serial_games_per_s": per_rate / span_s, "serial_p50_ms": pct(lat_s, 0.5),
                     "serial_p99_ms": pct(lat_s, 0.99),
                     "served_games_per_s": per_rate / done_at, "served_p50_ms": pct(lat_v, 0.5),
                     "served_p99_ms": pct(lat_v, 0.99)})
    for ar in arenas:
        ar.close()
    return {"requests_per_rate": per_rate, "game_scales": list(scales), "serial_capacity_games_per_s": cap,
            "rates": rows, "note": "latency = completion - arrival (host clock), credits delivered to host memory "
                                   "on both routes; server: continuous batching of games below 2^19 edges "
                                   "(64 slots, 16 GiB pool), larger games solved alone between slices"}


def cpu_parallel_baseline():
    """The paper's Algorithm 2 (OpenMP lifting sweeps from f = 0) on all host
    cores, on R-MAT scale 16 from the config-2 context's generator: context
    for the paper's multi-core CPU column (on the grid the sweeps from f = 0
    climb pseudo-polynomially and do not finish)."""
    import oracle
    from paper_1710_03647_gb300 import gen

    scale = 16
    a = gen.rmat_game(scale, 8, seed=CONTEXT_RMAT["seed"])
    t0 = time.perf_counter()
    _, st = oracle.sweep(a.n, a.row_ptr, a.col, a.w, a.owner_bits, threads=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    return {"value": st["edge_evals"] / dt, "unit": UNIT, "cores": st["threads"],
            "kind": "paper Algorithm 2 (parallel lifting sweeps)", "time_to_fixpoint_s": dt,
            "sweeps": st["sweeps"],
            "sample": f"R-MAT scale {scale} (n={a.n}, m={a.m}), f = 0 start, one full solve"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=WORKLOAD["side"], help="grid side of the headline (4000 = config 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the R-MAT scale-20 context (config 2)")
    ap.add_argument("--no-plain", action="store_true", help="skip the context solve without warm start")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched threshold-query comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-tune", action="store_true", help="time the default settings (no eg_autotune)")
    ap.add_argument("--settings", default=None,
                    help="headline launch settings as JSON ({\"local_windows\": 32, ...}), applied instead of "
                         "eg_autotune (e.g. to profile the tuned route without its search)")
    ap.add_argument("--no-scc", action="store_true", help="skip the SCC-ordered context solves")
    ap.add_argument("--batch-games", type=int, default=4096, help="games in the batched-vs-per-game comparison "
                    "(4096 = the full workload; 0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=512, help="requests per arrival rate (0 skips serving)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    import __graft_entry__

    __graft_entry__.build()
    from paper_1710_03647_gb300 import eg, gen

    side = args.side
    a = gen.grid_game(side, side, seed=WORKLOAD["seed"])
    bits = WORKLOAD["credit_bits"]
    if rank == 0:
        print(f"[bench] workload ready n={a.n} m={a.m}", file=sys.stderr, flush=True)
    s = bits // 8
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = torch.empty(a.n, dtype=torch.int64, device=dev)
    arena = eg.Arena(a)

    def step():
        _, st = eg.eg_solve_credit(arena.handle, bits, 1, 0, out, stream=stream.cuda_stream)
        return st

    # launch settings picked by the library's autotuner (timed solves, each
    # exact), outside the timed region; a fresh cache file, so it searches
    tuning = None
    given = json.loads(args.settings) if args.settings else None
    if given:
        unknown = set(given) - set(SETTING_KEYS)
        if unknown:
            raise SystemExit(f"--settings: unknown keys {sorted(unknown)}")
        arena.tune(**given)
    elif not args.no_tune:
        import tempfile

        t0 = time.perf_counter()
        with tempfile.TemporaryDirectory() as td:
            tuning = eg.eg_autotune(arena.handle, bits, 1, 0, os.path.join(td, "plans.jsonl"), max_solves=80)
        tuning["search_s"] = time.perf_counter() - t0

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    with ClockSampler(local) as clk:
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        clk.mark(True)
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xff)  # rewrite > L2 between steps (untimed)
                ev[k][0].record(stream)
            st = step()
            ev[k][1].record(stream)
            stats.append(st.as_dict())
        torch.cuda.synchronize()
        clk.mark(False)
    if pg:
        pg.barrier()
    step_ms = [b.elapsed_time(e) for b, e in ev]
    total_ms = sum(step_ms)
    relax = sum(x["relaxations"] for x in stats)
    settings = {k: tuning[k] for k in SETTING_KEYS} if tuning else dict(DEFAULT_SETTINGS, **(given or {}))
    launches = sum(launches_of(x, settings["sweeps"]) for x in stats)
    if pg:
        total_ms_max, relax_all = reduce_over_ranks(total_ms, relax, dev, pg)
    else:
        total_ms_max, relax_all = total_ms, float(relax)
    ok = all(x["status"] == 0 for x in stats)

    # dominant kernels: the lifting (dense sweeps and the persistent fixpoint);
    # the library times every lifting launch with CUDA events on the solve's
    # stream (phase_ms), summed here over all launches of all timed steps
    fix_ms = sum(x["fixpoint_ms"] for x in stats)
    n_launch = sum(x["phases"] for x in stats)
    wmax = int(np.abs(np.asarray(a.w, dtype=np.int64)).max())
    bytes_alg = sum(algorithmic_bytes(x, credit_bytes(x, wmax)) for x in stats)
    peak, peak_kind = peaks()
    achieved = bytes_alg / (fix_ms * 1e-3) / 1e9
    traffic = traffic_record(f"fixpoint_grid{side}_traffic.json", settings)

    # end to end through the public API: the arena from pinned host arrays
    # (eg_create copies them and builds the reverse CSR on the device), one
    # solve, the credits back to a pinned host array
    e2e = None
    if rank == 0 and not args.no_e2e:
        def pinned(x):
            return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()

        rp_h = pinned(np.asarray(a.row_ptr, dtype=np.int64))
        col_h, w_h = pinned(np.asarray(a.col, dtype=np.int32)), pinned(np.asarray(a.w, dtype=np.int32))
        ob_h = pinned(np.asarray(a.owner_bits, dtype=np.uint32).view(np.int32))
        host_out = torch.empty(a.n, dtype=torch.int64).pin_memory()
        e_times, e_relax, e_create = [], 0, []
        for k in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = eg.eg_create(a.n, a.m, rp_h, col_h, w_h, owner_bits=ob_h)
            for key, val in settings.items():  # the settings the timed steps ran with
                eg.eg_set_option(h, getattr(eg, "EG_OPT_" + key.upper()), int(val))
            t1 = time.perf_counter()
            _, st = eg.eg_solve_credit(h, bits, 1, 0, host_out)
            eg.eg_destroy(h)
            e_times.append(time.perf_counter() - t0)
            e_create.append(t1 - t0)
            e_relax += st.relaxations
        h2d = sum(t.numel() * t.element_size() for t in (rp_h, col_h, w_h, ob_h))
        e2e = {"value": e_relax / sum(e_times), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size() + 128),
               "ms_per_step": 1e3 * sum(e_times) / len(e_times),
               "eg_create_ms": 1e3 * statistics.median(e_create), "host_buffers": "pinned",
               "settings": "the timed steps' launch settings, set with eg_set_option on each new arena"}

    single = world == 1
    context = None
    rarena = None
    if single and not args.no_context:
        rarena, ra, context = rmat_context(eg, gen, torch, dev, stream, flush, plain_start=not args.no_plain,
                                           tune=not args.no_tune, scc=not args.no_scc)

    # 256 mean-payoff threshold queries on the R-MAT arena (w' = 256 w - k W,
    # k = -128..127, W = 100): one batched launch vs one solve per query
    thresholds = None
    if rarena is not None and not args.no_batch:
        ks = list(range(-128, 128))
        plan = eg.Plan(rarena.handle, len(ks), part=[0] * len(ks), w_scale=[256] * len(ks),
                       w_shift=[k * 100 for k in ks])
        bout = torch.empty(plan.total, dtype=torch.int64, device=dev)
        for _ in range(2):
            plan.run(bout, stream=stream.cuda_stream)
        bms, brelax = [], 0
        for _ in range(3):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            b0, b1 = ev_pair()
            b0.record(stream)
            _, bst = plan.run(bout, stream=stream.cuda_stream)
            b1.record(stream)
            torch.cuda.synchronize()
            bms.append(b0.elapsed_time(b1))
            brelax = bst.relaxations
        one = torch.empty(ra.n, dtype=torch.int64, device=dev)
        qms = []
        for k in ks:
            q0, q1 = ev_pair()
            q0.record(stream)
            eg.eg_solve_credit(rarena.handle, 64, 256, k * 100, one, stream=stream.cuda_stream)
            q1.record(stream)
            torch.cuda.synchronize()
            qms.append(q0.elapsed_time(q1))
        plan.close()
        bmed = statistics.median(bms)
        qms_sorted = sorted(qms)
        thresholds = {"queries": len(ks), "batched_ms": bmed, "batched_games_per_s": len(ks) / (bmed * 1e-3),
                      "batched_relaxations": brelax, "batched_p50_ms": bmed, "batched_p99_ms": max(bms),
                      "per_query_total_ms": sum(qms), "per_query_games_per_s": len(ks) / (sum(qms) * 1e-3),
                      "per_query_p50_ms": qms_sorted[len(qms) // 2],
                      "per_query_p99_ms": qms_sorted[min(len(qms) - 1, int(0.99 * len(qms)))],
                      "note": "batched: all queries in one persistent launch (CUDA graph); latency of every "
                              "query = the batch time"}
    if rarena is not None:
        rarena.close()

    batch = served = None
    if single and args.batch_games > 0:
        batch = batch_games(eg, gen, torch, dev, stream, args.batch_games, tune=not args.no_tune)
    if single and args.serve_requests > 0:
        served = serving(eg, gen, torch, dev, stream, args.serve_requests)

    if rank != 0:
        arena.close()
        if pg:
            pg.destroy_process_group()
        return
    g = golden(WORKLOAD["golden"]) if side == WORKLOAD["side"] else None
    oracle_ref = None
    if g:
        oracle_ref = {"time_to_fixpoint_s": g["oracle_seconds"], "edge_evaluations": g["oracle_lift_edge_evals"] +
                      g["oracle_pre_scans"], "route": "certified composition of Algorithm 1 runs, 1 thread "
                      "(Algorithm 1 with cap C alone would need ~1e14 lifts)", "trial": g["trial"],
                      "speedup": g["oracle_seconds"] * 1e3 / statistics.median(step_ms)}
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline()
    cpu_par = None if args.no_cpu_baseline or world > 1 else cpu_parallel_baseline()
    st0 = stats[-1]
    line = {
        "metric": METRIC, "value": relax_all / (total_ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["workload"] if side == WORKLOAD["side"] else f"grid{side}_s1",
                   "n": a.n, "m": a.m, "credit_bits": bits,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between steps (512 MiB write); arena and state exceed L2"},
        "all_exact": ok,
        "settings": "autotuned (eg_autotune)" if tuning else "given (--settings)" if given else "defaults",
        "launch_settings": settings,
        "tuning": tuning,
        "time_to_fixpoint_ms": statistics.median(step_ms),
        "oracle": oracle_ref,
        "rounds": st0["rounds"], "relaxations_per_step": st0["relaxations"], "lifts": st0["lifts"],
        "pushes": st0["pushes"], "trials": st0["trials"], "phases": st0["phase_list"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "k_sweep + k_fixpoint (the lifting kernels)",
                     "peak_kind": peak_kind,
                     "per": "step: every lifting launch of one solve (the dense sweeps and the fixpoint kernel of "
                            "the attempt and of each slice of the trials' lifts)",
                     "phases_per_step": n_launch / args.steps,
                     "algorithmic_bytes_per_step": bytes_alg / args.steps,
                     "kernel_ms_per_step": fix_ms / args.steps},
        "cpu_baseline": cpu,
        "cpu_parallel_baseline": cpu_par,
        "proven_player1": st0["seeded"],
        "rmat_context": context,
        "threshold_queries": thresholds,
        "batch_games": batch,
        "serving": served,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    arena.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
