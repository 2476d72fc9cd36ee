"""The N > 1 bench path on CPU: two gloo ranks, each a replica.  The job time
is the slowest rank's and the work the sum of the ranks' (no collective on the
data path; the reduction only combines timings)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)
        relax = 1000 * (rank + 1)
        got = bench.reduce_over_ranks(ms, relax, torch.device("cpu"), dist)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert results[r] == (20.0, 3000.0)


def test_reference_arm_non_zero_ranks_exit_quietly(capsys):
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(A, 2, 1)  # rank 1 does no work and prints nothing
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_the_contract_line(capsys, monkeypatch):
    import json

    import bench
    import oracle

    oracle.build()
    monkeypatch.setattr(bench, "SAMPLE_SIDE", 40)  # a small sample of the same generator

    class A:
        steps, warmup, gpus = 2, 1, 1

    bench.run_reference(A, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert "40x40" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
