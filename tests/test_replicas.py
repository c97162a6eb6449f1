"""The multi-GPU form of the benchmark is independent replicas (no data-path
collective): each rank runs the whole workload and the job's time is the
slowest rank's.  The host logic of that reduction is checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 100.0 + 50.0 * rank  # rank 1 is the slow replica
        t = bench.max_over_ranks(elapsed, dist, "cpu")
        out[rank] = (t, bench.whole_job_rate(1e9, world, t))
    finally:
        dist.destroy_process_group()


def test_replica_time_is_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == 150.0
    assert rate == pytest.approx(2e9 / 0.150)


def test_single_rank_passes_through():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(3e6, 1, 1000.0) == pytest.approx(3e6)
