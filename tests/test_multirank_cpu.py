"""The benchmark's multi-rank path on CPU (gloo, world size 2).

Each rank of `bench.py --gpus N` runs its own replica of the workload (the
path shards by independent surfaces, with no collective on the data path);
the timing is the maximum over ranks and the value is all ranks' units over
that time.  These helpers are exercised here with two gloo processes.
"""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [3.0, 5.0][rank]
        ms = bench.max_over_ranks(local_ms, torch.device("cpu"), world)
        rate = bench.whole_job_rate(1000, world, ms * 1e-3)
        dist.barrier()
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms, rate in res:
        assert ms == 5.0                       # slowest rank
        assert rate == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(2.5, None, 1) == 2.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
