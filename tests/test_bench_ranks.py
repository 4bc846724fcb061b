"""The multi-process path of bench.py on CPU: with two gloo ranks, every rank
gets the slowest rank's time, and the whole-job throughput counts every
rank's bytes over that time (replicas, weak scaling)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [120.0, 150.0][rank]
    got = bench.max_over_ranks(ms, world, torch.device("cpu"))
    value = bench.job_gbs(world, 1e9, 5, got)
    q.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 150.0  # the slower replica
        assert abs(value - 2 * 1e9 * 5 / 0.150 / 1e9) < 1e-9


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(42.0, 1, None) == 42.0
    assert abs(bench.job_gbs(1, 2e9, 4, 1000.0) - 8.0) < 1e-12
