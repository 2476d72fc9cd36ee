"""Thin ctypes binding of libeg.so (include/eg.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names (eg_create, eg_solve_credit, ...) and take numpy
arrays (host) or integer device addresses (e.g. torch.Tensor.data_ptr()).
The library is loaded from this package's _lib/ directory; if it is missing
the import of this module fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libeg.so")

EG_OK = 0
EG_PENDING = 1
EG_ERR_INVALID = -1
EG_ERR_NOT_TOTAL = -2
EG_ERR_OVERFLOW = -3
EG_ERR_OOM = -4
EG_ERR_CUDA = -5
EG_ERR_TIMEOUT = -6
EG_ERR_BUDGET = -7
EG_ERR_BUSY = -8
EG_TOP32 = np.iinfo(np.int32).max
EG_TOP64 = np.iinfo(np.int64).max
EG_INPUT_DEVICE = 1
EG_NOALLOC_MAX_VERTICES = 1 << 18

STATUS_NAMES = {0: "EG_OK", 1: "EG_PENDING", -1: "EG_ERR_INVALID", -2: "EG_ERR_NOT_TOTAL",
                -3: "EG_ERR_OVERFLOW", -4: "EG_ERR_OOM", -5: "EG_ERR_CUDA", -6: "EG_ERR_TIMEOUT",
                -7: "EG_ERR_BUDGET", -8: "EG_ERR_BUSY"}


EG_MAX_PHASES = 16
EG_PHASE_ATTEMPT = 0
EG_PHASE_DUAL = 1
EG_PHASE_CAPPED = 2
EG_PHASE_FINAL = 3
EG_PHASE_LEVEL = 4
PHASE_NAMES = {0: "attempt", 1: "dual", 2: "capped", 3: "final", 4: "level"}


class eg_stats(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int64), ("seeded", ctypes.c_int64), ("credit_bits", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rounds", ctypes.c_int64), ("lifts", ctypes.c_int64), ("pushes", ctypes.c_int64),
                ("relaxations", ctypes.c_int64), ("enqueues", ctypes.c_int64), ("ms", ctypes.c_double),
                ("fixpoint_ms", ctypes.c_double), ("cycle_jumps", ctypes.c_int64), ("phases", ctypes.c_int32),
                ("trials", ctypes.c_int32),
                ("phase_kind", ctypes.c_int32 * EG_MAX_PHASES), ("phase_cap", ctypes.c_int64 * EG_MAX_PHASES),
                ("phase_rounds", ctypes.c_int64 * EG_MAX_PHASES),
                ("phase_relaxations", ctypes.c_int64 * EG_MAX_PHASES),
                ("phase_ms", ctypes.c_double * EG_MAX_PHASES)]

    def phase_list(self) -> list[dict]:
        """The recorded fixpoint launches: kind, cap, rounds, relaxations, ms."""
        return [dict(kind=PHASE_NAMES.get(self.phase_kind[k], self.phase_kind[k]), cap=self.phase_cap[k],
                     rounds=self.phase_rounds[k], relaxations=self.phase_relaxations[k], ms=self.phase_ms[k])
                for k in range(self.phases)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("phase_")}
        d["phase_list"] = self.phase_list()
        return d


class eg_server_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "admitted", "solo", "taken_out", "completed", "refused",
                                               "slices", "idle_solo")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EG_SRV_FAIL_RESERVATIONS = 1
EG_SRV_IDLE_SOLO = 2


class eg_tuning(ctypes.Structure):
    _fields_ = [("local_windows", ctypes.c_int32), ("local_maxdeg", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("cap_certify", ctypes.c_int32),
                ("certify_after", ctypes.c_int64), ("dual_k", ctypes.c_int32), ("kick_rounds", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("chunk_edges", ctypes.c_int32),
                ("default_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double),
                ("solves", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("key", ctypes.c_char * 96)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["key"] = self.key.decode()
        return d


class EGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# exported symbol -> (restype, argtypes); the header's declarations
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
SIGNATURES = {
    "eg_create": (_I32, [_I64, _I64, _P, _P, _P, _P, _P, _P, _P, ctypes.c_uint32, ctypes.POINTER(_P)]),
    "eg_destroy": (_I32, [_P]),
    "eg_bound": (_I32, [_P, _I64, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "eg_solve_credit": (_I32, [_P, _I32, _I64, _I64, _P, ctypes.POINTER(eg_stats), _P, _I64]),
    "eg_set_option": (_I32, [_P, _I32, _I64]),
    "eg_set_parts": (_I32, [_P, _I32, _P]),
    "eg_plan_create": (_I32, [_P, _I32, _P, _P, _P, _I32, ctypes.POINTER(_P)]),
    "eg_plan_instance": (_I32, [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                ctypes.POINTER(_I32)]),
    "eg_plan_run": (_I32, [_P, _P, ctypes.POINTER(eg_stats), _P, _I64]),
    "eg_plan_destroy": (_I32, [_P]),
    "eg_solve_credit_noalloc": (_I32, [_P, _I32, _I64, _I64, _P, ctypes.POINTER(eg_stats), _P, _I64]),
    "eg_strategy": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P]),
    "eg_server_create": (_I32, [ctypes.c_size_t, _I32, ctypes.POINTER(_P)]),
    "eg_submit": (_I32, [_P, _P, _I32, _I64, _I64, ctypes.POINTER(ctypes.c_uint64)]),
    "eg_poll": (_I32, [_P, ctypes.c_uint64, _P, ctypes.POINTER(eg_stats)]),
    "eg_server_destroy": (_I32, [_P]),
    "eg_server_counters_get": (_I32, [_P, ctypes.POINTER(eg_server_counters)]),
    "eg_scc_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "eg_scc_levels": (_I32, [_P, _P, _P]),
    "eg_autotune": (_I32, [_P, _I32, _I64, _I64, ctypes.c_char_p, _I32, ctypes.POINTER(eg_tuning)]),
    "eg_plan_autotune": (_I32, [_P, ctypes.c_char_p, _I32, ctypes.POINTER(eg_tuning)]),
    "eg_server_set_option": (_I32, [_P, _I32, _I64]),
    "eg_last_error": (ctypes.c_char_p, []),
    "eg_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libeg.so and declares every entry point; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libeg.so not built at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def eg_last_error() -> str:
    return load().eg_last_error().decode()


def eg_version() -> str:
    return load().eg_version().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise EGError(rc, eg_last_error())
    return rc


def _addr(x, dtype):
    """Host numpy array (kept alive by the caller) or an int device address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    a = np.ascontiguousarray(x, dtype=dtype)
    if a is not x:
        raise TypeError(f"expected a contiguous {np.dtype(dtype)} array")
    return a.ctypes.data


def eg_create(n, m, row_ptr, col, w, rrow_ptr=None, rcol=None, rw=None, owner_bits=None, flags=0):
    """Returns an opaque arena handle (int).  Host arrays must already have
    the exact dtypes: int64 row_ptr, int32 col / w, uint32 owner_bits."""
    out = _P()
    rc = load().eg_create(n, m, _addr(row_ptr, np.int64), _addr(col, np.int32), _addr(w, np.int32),
                          _addr(rrow_ptr, np.int64), _addr(rcol, np.int32), _addr(rw, np.int32),
                          _addr(owner_bits, np.uint32), flags, ctypes.byref(out))
    _check(rc)
    return out.value


def eg_destroy(arena) -> None:
    _check(load().eg_destroy(arena))


def eg_bound(arena, w_scale: int = 1, w_shift: int = 0) -> tuple[int, int]:
    C, wm = _I64(), _I64()
    _check(load().eg_bound(arena, w_scale, w_shift, ctypes.byref(C), ctypes.byref(wm)))
    return C.value, wm.value


EG_OPT_LOCAL_WINDOWS = 1
EG_OPT_LOCAL_MAXDEG = 2
EG_OPT_WARM_START = 3
EG_OPT_SEED_MAX_PAIRS = 4
EG_OPT_GRAPH = 5
EG_OPT_CAP_CERTIFY = 6
EG_OPT_CERTIFY_AFTER = 7
EG_OPT_BLOCKS_PER_SM = 8
EG_OPT_WAIT_LIMIT_US = 9
EG_OPT_SCC_ORDER = 10
EG_OPT_DUAL_K = 11
EG_OPT_KICK_ROUNDS = 12
EG_OPT_CHUNK_EDGES = 13
EG_OPT_SWEEPS = 14


def eg_solve_credit_noalloc(arena, credit_bits, w_scale, w_shift, credits_out, stream=None, max_rounds=0,
                            raise_on_error=True):
    """Allocation-free solve; credits_out is a device buffer (address or
    tensor) of n elements of credit_bits (32 or 64).  Returns (status, eg_stats)."""
    st = eg_stats()
    rc = load().eg_solve_credit_noalloc(arena, credit_bits, w_scale, w_shift, _addr(credits_out, None),
                                        ctypes.byref(st), stream, max_rounds)
    if raise_on_error:
        _check(rc)
    return rc, st


def eg_strategy(arena, credit_bits, w_scale, w_shift, credits, succ_out=None, stream=None):
    """Player 0's winning successor per vertex (-1 where none) from least-EPM
    credits (numpy array or device tensor/address of credit_bits).  Returns
    succ_out (a new int32 numpy array if None)."""
    if isinstance(credits, np.ndarray):
        want = np.int32 if credit_bits == 32 else np.int64
        if credits.dtype != want or not credits.flags.c_contiguous:
            raise TypeError(f"credits must be a contiguous {np.dtype(want)} array")
        cptr = credits.ctypes.data
        n = credits.shape[0]
    else:
        cptr = _addr(credits, None)
        n = None
    if succ_out is None:
        if n is None:
            raise ValueError("succ_out is required with device credits")
        succ_out = np.empty(n, dtype=np.int32)
    optr = succ_out.ctypes.data if isinstance(succ_out, np.ndarray) else _addr(succ_out, None)
    _check(load().eg_strategy(arena, credit_bits, w_scale, w_shift, cptr, optr, stream))
    return succ_out


def eg_set_option(arena, option: int, value: int) -> None:
    _check(load().eg_set_option(arena, option, value))


def eg_solve_credit(arena, credit_bits, w_scale, w_shift, credits_out, stream=None, max_rounds=0,
                    raise_on_error=True):
    """credits_out: numpy array (host) or device address / tensor of the
    right width.  Returns (status, eg_stats)."""
    st = eg_stats()
    if isinstance(credits_out, np.ndarray):
        want = np.int32 if credit_bits == 32 else np.int64
        if credits_out.dtype != want or not credits_out.flags.c_contiguous:
            raise TypeError(f"credits_out must be a contiguous {np.dtype(want)} array")
        out_ptr = credits_out.ctypes.data
    else:
        out_ptr = _addr(credits_out, None)
    rc = load().eg_solve_credit(arena, credit_bits, w_scale, w_shift, out_ptr, ctypes.byref(st),
                                stream if stream is not None else None, max_rounds)
    if raise_on_error:
        _check(rc)
    return rc, st


class Arena:
    """Owns an eg_arena built from a gen.Arena-like object (host numpy arrays)."""

    def __init__(self, a, with_reverse=None):
        self.n, self.m = int(a.n), int(a.m)
        rev = with_reverse or (None, None, None)
        self.handle = eg_create(self.n, self.m, np.ascontiguousarray(a.row_ptr, np.int64),
                                np.ascontiguousarray(a.col, np.int32), np.ascontiguousarray(a.w, np.int32),
                                *rev, owner_bits=np.ascontiguousarray(a.owner_bits, np.uint32))

    def solve(self, credit_bits=0, w_scale=1, w_shift=0, stream=None, max_rounds=0):
        out = np.empty(self.n, dtype=np.int32 if credit_bits == 32 else np.int64)
        _, st = eg_solve_credit(self.handle, credit_bits, w_scale, w_shift, out, stream, max_rounds)
        return out, st

    def tune(self, local_windows=None, local_maxdeg=None, warm_start=None, seed_max_pairs=None, cap_certify=None,
             certify_after=None, blocks_per_sm=None, wait_limit_us=None, scc_order=None, dual_k=None,
             kick_rounds=None, chunk_edges=None, sweeps=None):
        for opt, val in ((EG_OPT_LOCAL_WINDOWS, local_windows), (EG_OPT_LOCAL_MAXDEG, local_maxdeg),
                         (EG_OPT_WARM_START, warm_start), (EG_OPT_SEED_MAX_PAIRS, seed_max_pairs),
                         (EG_OPT_CAP_CERTIFY, cap_certify), (EG_OPT_CERTIFY_AFTER, certify_after),
                         (EG_OPT_BLOCKS_PER_SM, blocks_per_sm), (EG_OPT_WAIT_LIMIT_US, wait_limit_us),
                         (EG_OPT_SCC_ORDER, scc_order), (EG_OPT_DUAL_K, dual_k),
                         (EG_OPT_KICK_ROUNDS, kick_rounds), (EG_OPT_CHUNK_EDGES, chunk_edges),
                         (EG_OPT_SWEEPS, sweeps)):
            if val is not None:
                eg_set_option(self.handle, opt, int(val))

    def bound(self, w_scale=1, w_shift=0):
        return eg_bound(self.handle, w_scale, w_shift)

    def close(self):
        if self.handle:
            eg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eg_set_parts(arena, part_ptr) -> None:
    pp = np.ascontiguousarray(part_ptr, dtype=np.int64)
    _check(load().eg_set_parts(arena, pp.shape[0] - 1, pp.ctypes.data))


def pack_games(games):
    """Disjoint union of arenas (objects with n, row_ptr, col, w, owner_bits):
    returns (n, row_ptr, col, w, owner_bits, part_ptr) with game k's vertex v
    at part_ptr[k] + v."""
    ns = [int(g.n) for g in games]
    part_ptr = np.zeros(len(games) + 1, dtype=np.int64)
    np.cumsum(ns, out=part_ptr[1:])
    ms = [int(g.row_ptr[-1]) for g in games]
    eoff = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    n = int(part_ptr[-1])
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(int(eoff[-1]), dtype=np.int32)
    w = np.empty(int(eoff[-1]), dtype=np.int32)
    own = np.zeros(n, dtype=bool)
    for k, g in enumerate(games):
        a, b = int(part_ptr[k]), int(part_ptr[k + 1])
        row_ptr[a:b] = np.asarray(g.row_ptr[:-1], dtype=np.int64) + eoff[k]
        col[eoff[k]:eoff[k + 1]] = np.asarray(g.col, dtype=np.int64) + a
        w[eoff[k]:eoff[k + 1]] = g.w
        idx = np.arange(g.n)
        own[a:b] = (np.asarray(g.owner_bits, dtype=np.uint32)[idx >> 5] >> (idx & 31).astype(np.uint32)) & 1
    row_ptr[n] = eoff[-1]
    words = (n + 31) // 32
    padded = np.zeros(words * 32, dtype=np.uint64)
    padded[:n] = own
    owner_bits = (padded.reshape(words, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    return n, row_ptr, col, w, owner_bits, part_ptr


class Plan:
    """A batched solve: count instances (game part[i] under w' = scale*w - shift)."""

    def __init__(self, arena_handle, count, part=None, w_scale=None, w_shift=None, credit_bits=0):
        self._keep = []

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data

        out = _P()
        _check(load().eg_plan_create(arena_handle, count, arr(part, np.int32), arr(w_scale, np.int64),
                                     arr(w_shift, np.int64), credit_bits, ctypes.byref(out)))
        self.handle = out.value
        self.count = count
        self.credit_bits = credit_bits
        self.total = sum(self.instance(i)[1] for i in range(count))

    def instance(self, i):
        """(offset, n, C, bits the instance alone needs)"""
        off, n, C, b = _I64(), _I64(), _I64(), _I32()
        _check(load().eg_plan_instance(self.handle, i, ctypes.byref(off), ctypes.byref(n), ctypes.byref(C),
                                       ctypes.byref(b)))
        return off.value, n.value, C.value, b.value

    def run(self, out=None, stream=None, max_rounds=0, raise_on_error=True):
        if out is None:
            out = np.empty(self.total, dtype=np.int32 if self.credit_bits == 32 else np.int64)
        st = eg_stats()
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else _addr(out, None)
        rc = load().eg_plan_run(self.handle, ptr, ctypes.byref(st), stream, max_rounds)
        if raise_on_error:
            _check(rc)
        return out, st

    def close(self):
        if self.handle:
            _check(load().eg_plan_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eg_server_create(device_mem_budget: int, max_batch: int):
    out = _P()
    _check(load().eg_server_create(device_mem_budget, max_batch, ctypes.byref(out)))
    return out.value


def eg_submit(server, arena, credit_bits=0, w_scale=1, w_shift=0) -> int:
    t = ctypes.c_uint64()
    _check(load().eg_submit(server, arena, credit_bits, w_scale, w_shift, ctypes.byref(t)))
    return t.value


def eg_poll(server, ticket, credits_out=None):
    """(status, eg_stats); status EG_PENDING until the request is done.
    Errors of the request come back as the status (not raised)."""
    st = eg_stats()
    ptr = None
    if credits_out is not None:
        ptr = credits_out.ctypes.data if isinstance(credits_out, np.ndarray) else _addr(credits_out, None)
    rc = load().eg_poll(server, ticket, ptr, ctypes.byref(st))
    return rc, st


def eg_server_destroy(server) -> None:
    _check(load().eg_server_destroy(server))


def eg_server_counters_get(server) -> dict:
    c = eg_server_counters()
    _check(load().eg_server_counters_get(server, ctypes.byref(c)))
    return c.as_dict()


def eg_server_set_option(server, option: int, value: int) -> None:
    _check(load().eg_server_set_option(server, option, value))


def eg_autotune(arena, credit_bits=0, w_scale=1, w_shift=0, cache_path=None, max_solves=0) -> dict:
    """Tunes the arena's launch settings (see eg.h); returns the eg_tuning fields."""
    t = eg_tuning()
    path = cache_path.encode() if cache_path else None
    _check(load().eg_autotune(arena, credit_bits, w_scale, w_shift, path, max_solves, ctypes.byref(t)))
    return t.as_dict()


def eg_plan_autotune(plan, cache_path=None, max_solves=0) -> dict:
    t = eg_tuning()
    path = cache_path.encode() if cache_path else None
    handle = plan.handle if isinstance(plan, Plan) else plan
    _check(load().eg_plan_autotune(handle, path, max_solves, ctypes.byref(t)))
    return t.as_dict()


def eg_scc_info(arena) -> dict:
    """Components, topological levels and kernel passes of the arena's condensation."""
    c, l, p = _I64(), _I64(), _I64()
    _check(load().eg_scc_info(arena, ctypes.byref(c), ctypes.byref(l), ctypes.byref(p)))
    return {"components": c.value, "levels": l.value, "passes": p.value}


def eg_scc_levels(arena, n):
    """(level, component) int32 arrays of the arena's n vertices."""
    level = np.empty(n, dtype=np.int32)
    comp = np.empty(n, dtype=np.int32)
    _check(load().eg_scc_levels(arena, level.ctypes.data, comp.ctypes.data))
    return level, comp
