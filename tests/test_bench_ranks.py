"""bench.py's multi-GPU arithmetic on CPU: N replicas (one process per GPU)
each time their own frames; the job's time is the slowest rank's, taken with
an all-reduce over the process group, and the throughput counts every rank's
frames.  Two gloo ranks on 127.0.0.1 stand in for two GPUs."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(ms_by_rank[rank], world, "cpu")
    out.put((rank, slowest, bench.replica_rate(slowest, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    ms_by_rank = [2.0, 2.5]
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms_by_rank, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for _, slowest, rate in res:
        assert slowest == 2.5
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.replica_rate(4.0, 1, 64) == pytest.approx(16000.0)
