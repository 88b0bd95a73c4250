"""The benchmark's multi-rank path (independent replicas, one per GPU) on CPU:
two gloo ranks report different times; the job time is the slowest rank's and
the throughput counts every rank's work."""
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


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    ms, qps = bench.combine_ranks(dist, torch.device("cpu"), local_ms, 1_000_000, ws)
    out[rank] = (ms, qps)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_max_time_and_sum_work():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(ws):
        ms, qps = out[r]
        assert ms == 200.0
        assert qps == pytest.approx(2 * 1_000_000 / 0.2)


def test_single_rank_needs_no_collective():
    import bench
    ms, qps = bench.combine_ranks(None, None, 50.0, 1000, 1)
    assert ms == 50.0 and qps == pytest.approx(20000.0)
