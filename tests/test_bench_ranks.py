"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks run
replicas of different speed; every rank must take the slowest rank's time,
and the whole-job rate counts the nodes of both replicas over that time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(times[rank], dist, device="cpu")
        out[rank] = (t, bench.whole_job_mlups(1000, 10, world, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    world, port = 2, _free_port()
    times = [0.5, 0.8]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        got = dict(out)
    for r in range(world):
        t, v = got[r]
        assert t == pytest.approx(0.8)
        assert v == pytest.approx(1000 * 10 * 2 / 0.8 / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_mlups(10, 2, 1, 0.5) == pytest.approx(4e-5)
