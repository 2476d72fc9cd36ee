"""Seeded synthetic energy-game arenas.

This module only draws inputs: graph shapes, ownership and integer edge
weights.  It contains none of the solver's arithmetic (no bound, no credit
operator), so both the CUDA path and the CPU oracle can be fed from it.

Randomness comes from a counter-based splitmix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream (seed, tag) is mix(key + (i + 1) * 0x9E3779B97F4A7C15) with
key = mix(seed * 0x100000001B3 + tag).  The same (seed, tag, i) gives the
same number on every machine and numpy version.

An arena is the game graph of the paper's Sec. 2 (a total weighted graph
with an owner partition): forward CSR (row_ptr int64 of n+1, col int32,
w int32) plus an ownership bitmap, bit v of word v // 32 set iff v is a
player-1 vertex.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream identified by (seed, tag)."""

    def __init__(self, seed: int, tag: int):
        with np.errstate(over="ignore"):
            k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.uint64(0x100000001B3) + np.uint64(tag)
        self.key = _mix(np.array([k], dtype=np.uint64))[0]

    def u64(self, count: int, offset: int = 0) -> np.ndarray:
        idx = np.arange(offset + 1, offset + 1 + count, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _GOLDEN)

    def below(self, count: int, bound, offset: int = 0) -> np.ndarray:
        """Integers in [0, bound) by the multiply-shift map on the top 32 bits.

        `bound` may be a scalar or an array (one bound per draw), < 2**32.
        """
        hi = self.u64(count, offset) >> np.uint64(32)
        b = np.asarray(bound, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return ((hi * b) >> np.uint64(32)).astype(np.int64)

    def unit(self, count: int, offset: int = 0) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, count: int, lo, hi, offset: int = 0) -> np.ndarray:
        """Integers uniform in the closed range [lo, hi] (scalars or arrays)."""
        lo = np.asarray(lo, dtype=np.int64)
        hi = np.asarray(hi, dtype=np.int64)
        return lo + self.below(count, hi - lo + 1, offset)


@dataclasses.dataclass
class Arena:
    """One game arena in forward CSR form (host numpy arrays)."""

    n: int
    row_ptr: np.ndarray  # int64, n + 1
    col: np.ndarray  # int32, m
    w: np.ndarray  # int32, m
    owner_bits: np.ndarray  # uint32, ceil(n / 32); bit set <=> player 1
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def owner(self) -> np.ndarray:
        """Boolean array, True where the vertex belongs to player 1."""
        return unpack_owner(self.owner_bits, self.n)

    def with_weights(self, w: np.ndarray, name: str | None = None) -> "Arena":
        return Arena(self.n, self.row_ptr, self.col, np.ascontiguousarray(w, dtype=np.int32),
                     self.owner_bits, self.name if name is None else name)


def pack_owner(is_p1: np.ndarray) -> np.ndarray:
    is_p1 = np.asarray(is_p1, dtype=bool)
    n = is_p1.shape[0]
    words = (n + 31) // 32
    padded = np.zeros(words * 32, dtype=np.uint64)
    padded[:n] = is_p1
    shifts = np.arange(32, dtype=np.uint64)
    packed = (padded.reshape(words, 32) << shifts).sum(axis=1)
    return packed.astype(np.uint32)


def unpack_owner(bits: np.ndarray, n: int) -> np.ndarray:
    bits = np.asarray(bits, dtype=np.uint32)
    idx = np.arange(n)
    return ((bits[idx >> 5] >> (idx & 31).astype(np.uint32)) & 1).astype(bool)


def _owners(n: int, seed: int, p1: float = 0.5) -> np.ndarray:
    return pack_owner(Stream(seed, 1).unit(n) < p1)


def _csr_from_rows(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Stable CSR build: edges keep their relative order within a row."""
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, dst[order].astype(np.int32)


def _distinct_successors(n: int, deg: np.ndarray, stream: Stream) -> tuple[np.ndarray, np.ndarray]:
    """For vertex v, deg[v] distinct successors drawn uniformly from V minus {v}.

    Duplicates inside a row are redrawn (the later slot of a pair) from fresh
    counters until none remain.  Requires deg[v] <= n - 1.
    """
    deg = np.asarray(deg, dtype=np.int64)
    if n > 1 and int(deg.max(initial=0)) > n - 1:
        raise ValueError("out-degree larger than n - 1")
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    m = src.shape[0]
    slots = np.arange(m, dtype=np.int64)
    dst = np.empty(m, dtype=np.int64)
    todo = slots
    offset = 0
    while todo.shape[0]:
        x = stream.below(todo.shape[0], n - 1, offset)
        offset += todo.shape[0]
        x = x + (x >= src[todo])
        dst[todo] = x
        key = src * n + dst
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(m, dtype=bool)
        dup[order[1:][ks[1:] == ks[:-1]]] = True
        todo = slots[dup]
    return src, dst


def uniform_game(n: int, deg: int = 4, wlo: int = -10, whi: int = 10, seed: int = 1,
                 name: str = "") -> Arena:
    """Each vertex gets exactly `deg` distinct uniform successors other than itself;
    ownership Bernoulli(0.5); weights uniform in [wlo, whi]."""
    degs = np.full(n, deg, dtype=np.int64)
    src, dst = _distinct_successors(n, degs, Stream(seed, 2))
    row_ptr, col = _csr_from_rows(n, src, dst)
    w = Stream(seed, 3).integers(col.shape[0], wlo, whi).astype(np.int32)
    return Arena(n, row_ptr, col, w, _owners(n, seed), name or f"uniform_n{n}_d{deg}_w{whi}_s{seed}")


def varied_game(n: int, dlo: int, dhi: int, W: int, seed: int, name: str = "") -> Arena:
    """Out-degree uniform in [dlo, dhi] per vertex (distinct successors other
    than the vertex), weights uniform in [-W, W], ownership Bernoulli(0.5)."""
    dhi_eff = min(dhi, n - 1)
    dlo_eff = min(dlo, dhi_eff)
    degs = Stream(seed, 4).integers(n, dlo_eff, dhi_eff)
    src, dst = _distinct_successors(n, degs, Stream(seed, 2))
    row_ptr, col = _csr_from_rows(n, src, dst)
    w = Stream(seed, 3).integers(col.shape[0], -W, W).astype(np.int32)
    return Arena(n, row_ptr, col, w, _owners(n, seed), name or f"varied_n{n}_d{dlo}-{dhi}_W{W}_s{seed}")


def rmat_game(scale: int = 20, edge_factor: int = 8, abcd=(0.57, 0.19, 0.19, 0.05),
              wlo: int = -100, whi: int = 100, seed: int = 1, name: str = "") -> Arena:
    """R-MAT arena: edge_factor * 2**scale draws of the recursive quadrant
    process (Chakrabarti, Zhan, Faloutsos 2004), self-loops and repeated pairs
    dropped, every vertex left without a successor given one uniform successor
    other than itself, no relabelling; weights uniform in [wlo, whi]."""
    n = 1 << scale
    draws = edge_factor * n
    a, b, c, _ = abcd
    s = Stream(seed, 5)
    src = np.zeros(draws, dtype=np.int64)
    dst = np.zeros(draws, dtype=np.int64)
    for level in range(scale):
        u = s.unit(draws, level * draws)
        rbit = (u >= a + b).astype(np.int64)
        cbit = (((u >= a) & (u < a + b)) | (u >= a + b + c)).astype(np.int64)
        src = (src << 1) | rbit
        dst = (dst << 1) | cbit
    keep = src != dst
    key = np.unique(src[keep] * n + dst[keep])
    src, dst = key // n, key % n
    outdeg = np.bincount(src, minlength=n)
    lonely = np.nonzero(outdeg == 0)[0]
    if lonely.shape[0]:
        x = Stream(seed, 6).below(lonely.shape[0], n - 1)
        x = x + (x >= lonely)
        key = np.concatenate([key, lonely * n + x])
        key.sort()
        src, dst = key // n, key % n
    row_ptr, col = _csr_from_rows(n, src, dst)
    w = Stream(seed, 3).integers(col.shape[0], wlo, whi).astype(np.int32)
    return Arena(n, row_ptr, col, w, _owners(n, seed), name or f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def grid_game(rows: int = 4000, cols: int = 4000, long_frac: float = 0.01, neg_p: float = 0.4,
              wneg: int = 1000, wpos: int = 1000, seed: int = 1, name: str = "") -> Arena:
    """Road-like arena: directed edges to the 4 grid neighbours (up, down,
    left, right where they exist) plus round(long_frac * grid edges) long
    edges with uniform source and uniform target other than the source.
    A weight is negative with probability neg_p, uniform in [-wneg, -1],
    otherwise uniform in [0, wpos]."""
    n = rows * cols
    vid = np.arange(n, dtype=np.int64)
    r, c = vid // cols, vid % cols
    parts_src, parts_dst = [], []
    for dr, dc in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (r + dr >= 0) & (r + dr < rows) & (c + dc >= 0) & (c + dc < cols)
        parts_src.append(vid[ok])
        parts_dst.append(vid[ok] + dr * cols + dc)
    gsrc = np.concatenate(parts_src)
    gdst = np.concatenate(parts_dst)
    # stable sort keeps up/down/left/right order inside a row
    order = np.argsort(gsrc, kind="stable")
    gsrc, gdst = gsrc[order], gdst[order]
    nlong = int(round(long_frac * gsrc.shape[0]))
    s = Stream(seed, 7)
    lsrc = s.below(nlong, n, 0)
    ldst = s.below(nlong, n - 1, nlong)
    ldst = ldst + (ldst >= lsrc)
    src = np.concatenate([gsrc, lsrc])
    dst = np.concatenate([gdst, ldst])
    row_ptr, col = _csr_from_rows(n, src, dst)
    m = col.shape[0]
    neg = Stream(seed, 8).unit(m) < neg_p
    mag_neg = Stream(seed, 9).integers(m, 1, wneg)
    mag_pos = Stream(seed, 10).integers(m, 0, wpos)
    w = np.where(neg, -mag_neg, mag_pos).astype(np.int32)
    return Arena(n, row_ptr, col, w, _owners(n, seed), name or f"grid_{rows}x{cols}_s{seed}")


def tiny_game(n: int, max_deg: int = 3, wlo: int = -4, whi: int = 4, seed: int = 1,
              self_loops: bool = True, p1: float = 0.5) -> Arena:
    """Small arena for exhaustive checks: out-degree uniform in [1, max_deg],
    successors uniform over all of V (self-loops and repeated targets
    allowed when `self_loops`), weights uniform in [wlo, whi]."""
    s = Stream(seed, 11)
    degs = 1 + s.below(n, max_deg)
    m = int(degs.sum())
    src = np.repeat(np.arange(n, dtype=np.int64), degs)
    if self_loops:
        dst = Stream(seed, 12).below(m, n)
    else:
        x = Stream(seed, 12).below(m, max(n - 1, 1))
        dst = x + (x >= src) if n > 1 else x
    row_ptr, col = _csr_from_rows(n, src, dst)
    w = Stream(seed, 13).integers(m, wlo, whi).astype(np.int32)
    return Arena(n, row_ptr, col, w, pack_owner(Stream(seed, 14).unit(n) < p1), f"tiny_n{n}_s{seed}")


def batch_shapes(count: int = 4096, nlo: int = 1000, nhi: int = 200000, Wlo: int = 10,
                 Whi: int = 10000, seed: int = 1) -> list[tuple[int, int]]:
    """(n, W) for a batch of uneven games: n and W log-uniform in their ranges."""
    un = Stream(seed, 15).unit(count)
    uw = Stream(seed, 16).unit(count)
    ns = np.floor(np.exp(math.log(nlo) + un * (math.log(nhi) - math.log(nlo)))).astype(np.int64)
    Ws = np.rint(np.exp(math.log(Wlo) + uw * (math.log(Whi) - math.log(Wlo)))).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(ns, Ws)]


def batch_game(i: int, n: int, W: int, seed: int = 1, dlo: int = 2, dhi: int = 16) -> Arena:
    """Game i of a batch: out-degree uniform in [dlo, dhi], weights in [-W, W]."""
    return varied_game(n, dlo, dhi, W, seed * 1000003 + i, name=f"batch{i}_n{n}_W{W}")


def threshold_weights(w: np.ndarray, k: int, W: int, scale: int = 256) -> np.ndarray:
    """Shifted weights scale * w - k * W of a mean-payoff threshold query
    (an integer restatement of the threshold k / scale * W), as int64."""
    return np.asarray(w, dtype=np.int64) * scale - np.int64(k) * W


def config(idx: int, seed: int = 1, shrink: int = 1) -> Arena:
    """The paper-scale synthetic workloads: 1 uniform 1k game, 2 R-MAT scale 20,
    3 4000x4000 road-like grid.  `shrink` > 1 scales sizes down for quick runs."""
    if idx == 1:
        return uniform_game(1000 // shrink if shrink > 1 else 1000, 4, -10, 10, seed, name=f"uniform1k_s{seed}")
    if idx == 2:
        scale = 20 - int(round(math.log2(shrink))) if shrink > 1 else 20
        return rmat_game(scale, 8, seed=seed, name=f"rmat{scale}_s{seed}")
    if idx == 3:
        side = 4000 // int(round(math.sqrt(shrink))) if shrink > 1 else 4000
        return grid_game(side, side, seed=seed, name=f"grid{side}_s{seed}")
    raise ValueError(idx)


def _batch_game_job(args) -> Arena:
    i, n, W, seed = args
    return batch_game(i, n, W, seed)


def batch_games(count: int = 4096, seed: int = 1, workers: int = 16) -> list[Arena]:
    """The `count` games of the uneven batch (batch_shapes, batch_game).  Large
    batches are drawn by a pool of spawned processes (spawned, so that no
    CUDA state of the caller is forked); the result does not depend on it."""
    import multiprocessing as mp
    import os

    jobs = [(i, n, W, seed) for i, (n, W) in enumerate(batch_shapes(count, seed=seed))]
    workers = min(workers, os.cpu_count() or 1)
    if len(jobs) <= 64 or workers <= 1:
        return [_batch_game_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_batch_game_job, jobs, chunksize=8)
