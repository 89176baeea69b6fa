"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks, max-over-ranks time and the
whole-job value (each rank runs an independent replica of the step; no data-path collective)."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms)
        value = bench.job_value(1000.0, world, slowest)
        out[rank] = (slowest, value)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import random

    port = 29500 + random.randint(0, 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 150.0
    assert abs(value - 2 * 1000.0 / 0.150) < 1e-6


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_value(10.0, 1, 1000.0) == 10.0
