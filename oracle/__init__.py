"""CPU oracle for the energy-game initial credit problem (arXiv 1710.03647).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may use this package; the CUDA product path never does.  It shares
no code with the CUDA solver.  `oracle.c` holds the arithmetic:

  bound(...)        M_G of Sec. 3.1
  solve(...)        Algorithm 1 of Sec. 3.1 (FIFO worklist with counters)
  brute_force(...)  Lemma "EGcycles" by strategy enumeration + Bellman-Ford
  check(...)        least-EPM equations of Def. "EPM" / "Lifting Operator"

`sweep.c` (its own library, built with OpenMP) is the paper's Algorithm 2,
the multi-core CPU baseline the benchmark times as context:

  sweep(...)        parallel in-place lifting sweeps from f = 0

Credits are int64 numpy arrays with TOP = INT64_MAX.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

TOP = np.iinfo(np.int64).max
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_SWEEP_SRC = os.path.join(_HERE, "sweep.c")
_SWEEP_LIB = os.path.join(_LIB_DIR, "liboracle_sweep.so")
_lib = None
_sweep_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (and sweep.c, with OpenMP) into shared libraries
    with the host C compiler."""
    for src, lib, extra in ((_SRC, _LIB, []), (_SWEEP_SRC, _SWEEP_LIB, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            os.makedirs(_LIB_DIR, exist_ok=True)
            tmp = lib + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", *extra, "-o", tmp, src]
            if subprocess.run(cmd, capture_output=True).returncode != 0:
                if not extra:
                    subprocess.check_call(cmd)
                # no OpenMP here: the sweep baseline builds single-threaded
                # (it reports the threads it used)
                subprocess.check_call([c for c in cmd if c not in extra])
            os.replace(tmp, lib)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_bound.restype = i64
        lib.oracle_bound.argtypes = [i64, p, p]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [i64, p, p, p, p, i64, i64, p, p]
        lib.oracle_brute_force.restype = ctypes.c_int
        lib.oracle_brute_force.argtypes = [i64, p, p, p, p, i64, p]
        lib.oracle_check.restype = ctypes.c_int
        lib.oracle_check.argtypes = [i64, p, p, p, p, i64, p, p]
        _lib = lib
    return _lib


def _arrays(row_ptr, col, w, owner_bits):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int64)
    owner_bits = np.ascontiguousarray(owner_bits, dtype=np.uint32)
    if owner_bits.size == 0:
        owner_bits = np.zeros(1, dtype=np.uint32)
    return row_ptr, col, w, owner_bits


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleError(RuntimeError):
    pass


def bound(n: int, row_ptr, w) -> int:
    """M_G = sum_v max(0, max over out-edges of -w)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.int64)
    return int(_load().oracle_bound(n, _ptr(row_ptr), _ptr(w) if w.size else None))


def solve(n: int, row_ptr, col, w, owner_bits, C: int | None = None, max_lifts: int = 0):
    """Algorithm 1.  Returns (f int64[n] with TOP, stats dict)."""
    row_ptr, col, w, owner_bits = _arrays(row_ptr, col, w, owner_bits)
    if C is None:
        C = bound(n, row_ptr, w)
    f = np.zeros(max(n, 1), dtype=np.int64)
    st = np.zeros(4, dtype=np.int64)
    rc = _load().oracle_solve(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(owner_bits), C, max_lifts,
                              _ptr(f), _ptr(st))
    if rc == 1:
        raise OracleError("arena is not total: a vertex has no successor")
    if rc == 2:
        raise OracleError(f"lift budget of {max_lifts} exhausted")
    if rc != 0:
        raise OracleError(f"oracle_solve failed with {rc}")
    stats = dict(C=C, lifts=int(st[0]), lift_edge_evals=int(st[1]), pre_scans=int(st[2]),
                 recount_evals=int(st[3]))
    return f[:n], stats


def brute_force(n: int, row_ptr, col, w, owner_bits, max_strategies: int = 1 << 20):
    """Minimum credits by exhaustive strategy enumeration (tiny arenas only)."""
    row_ptr, col, w, owner_bits = _arrays(row_ptr, col, w, owner_bits)
    c = np.zeros(max(n, 1), dtype=np.int64)
    rc = _load().oracle_brute_force(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(owner_bits),
                                    max_strategies, _ptr(c))
    if rc == 1:
        raise OracleError("arena is not total: a vertex has no successor")
    if rc == 2:
        raise OracleError("too many strategies for brute force")
    if rc != 0:
        raise OracleError(f"oracle_brute_force failed with {rc}")
    return c[:n]


def check(n: int, row_ptr, col, w, owner_bits, f, C: int | None = None):
    """(code, vertex): 0 if f is a fixpoint of every lift within {0..C} u {TOP}."""
    row_ptr, col, w, owner_bits = _arrays(row_ptr, col, w, owner_bits)
    if C is None:
        C = bound(n, row_ptr, w)
    f = np.ascontiguousarray(f, dtype=np.int64)
    bad = np.zeros(1, dtype=np.int64)
    rc = _load().oracle_check(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(owner_bits), C, _ptr(f),
                              _ptr(bad))
    return int(rc), int(bad[0])


def _load_sweep():
    global _sweep_lib
    if _sweep_lib is None:
        build()
        lib = ctypes.CDLL(_SWEEP_LIB)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_sweep.restype = ctypes.c_int
        lib.oracle_sweep.argtypes = [i64, p, p, p, p, i64, i64, ctypes.c_int, p, p]
        _sweep_lib = lib
    return _sweep_lib


def sweep(n: int, row_ptr, col, w, owner_bits, C: int | None = None, max_sweeps: int = 0, threads: int = 0):
    """Algorithm 2 (parallel sweeps).  Returns (f int64[n] with TOP, stats dict)."""
    row_ptr, col, w, owner_bits = _arrays(row_ptr, col, w, owner_bits)
    if C is None:
        C = bound(n, row_ptr, w)
    f = np.zeros(max(n, 1), dtype=np.int64)
    st = np.zeros(3, dtype=np.int64)
    rc = _load_sweep().oracle_sweep(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(owner_bits), C, max_sweeps,
                                    threads, _ptr(f), _ptr(st))
    if rc == 1:
        raise OracleError("arena is not total: a vertex has no successor")
    if rc == 2:
        raise OracleError(f"sweep budget of {max_sweeps} exhausted")
    return f[:n], dict(C=C, sweeps=int(st[0]), edge_evals=int(st[1]), threads=int(st[2]))


def certified_solve(n: int, row_ptr, col, w, owner_bits, C: int | None = None, cap_mult: int = 4,
                    trials: int = 8, log=None):
    """The least EPM by certified trial caps, built from Algorithm 1 alone.

    Two facts, each pinned by brute force in the oracle's tests, let capped
    runs of Algorithm 1 decide a game whose cap-C run would climb for hours:

      (dual)   in the game with weights -(K w + 1) (K >= 1) and the owners
               swapped, a vertex whose least fixpoint under any cap is
               finite is won by player 1 in the original game: player 1
               then has a positional strategy that keeps every cycle of the
               play at K w(c) + |c| <= 0, so w(c) < 0 (Lemma "EGcycles");
      (capped) the least fixpoint under a cap B < C is pointwise at or above
               the one under C; if every vertex is finite under B or proven
               lost by (dual), every finite credit is at most B, and a cap
               at or above the largest finite credit gives the same least
               fixpoint as C (Sec. 3.1 uses M_G only as an upper bound).

    Trial k runs Algorithm 1 on the dual (K = 8^(k+1), at most n + 1, cap
    (K + 1) B) and on the game with cap B = cap_mult * max|w| * 4^k, each
    from f = 0, and stops at the first trial that decides every vertex.
    If no trial does, the game is solved with cap C.  Each run starts from
    zero, so the result does not depend on the trial schedule: it is the
    unique least EPM.  Returns (f, stats) like solve(); stats adds the
    deciding trial (-1: cap C), its B and K, and the summed work counters.
    """
    row_ptr, col, w, owner_bits = _arrays(row_ptr, col, w, owner_bits)
    if C is None:
        C = bound(n, row_ptr, w)
    maxw = max(1, int(np.abs(w).max()) if w.size else 1)
    dual_owner = np.ascontiguousarray(~owner_bits, dtype=np.uint32)
    lim = 1 << 61
    tot = dict(lifts=0, lift_edge_evals=0, pre_scans=0, recount_evals=0)

    def add(st):
        for k in tot:
            tot[k] += st[k]

    lost = np.zeros(n, dtype=bool)
    B, K = cap_mult * maxw, min(8, n + 1)
    for k in range(trials):
        if B >= C or K * (maxw + 1) > lim or (K + 1) * B > lim:
            break
        wd = -(np.int64(K) * w) - 1
        fd, st = solve(n, row_ptr, col, wd, dual_owner, C=(K + 1) * B)
        add(st)
        lost |= fd != TOP
        fg, st = solve(n, row_ptr, col, w, owner_bits, C=B)
        add(st)
        decided = (fg != TOP) | lost
        if log:
            log(f"trial {k}: B={B} K={K} undecided={int((~decided).sum())}")
        if decided.all():
            return fg, dict(C=C, trial=k, B=B, K=K, **tot)
        B, K = B * 4, min(K * 8, n + 1)
    f, st = solve(n, row_ptr, col, w, owner_bits, C=C)
    add(st)
    return f, dict(C=C, trial=-1, B=C, K=0, **tot)
