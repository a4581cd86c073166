"""The benchmark's multi-GPU bookkeeping on CPU ranks (gloo, world size 2):
every ray is independent, so ranks shard frames with no collective on the data
path; the only exchange is the slowest rank's step time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 2.0 + rank  # rank 1 is slower
        m = bench.max_over_ranks(step_ms)
        out[rank] = (m, bench.whole_job_rate(5, m, world))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step_and_sum_the_work():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        m, rate = out[rank]
        assert m == 3.0
        assert abs(rate - 2 * 5 / 3.0e-3) < 1e-6


def test_single_process_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_rate(5, 2.0, 1) == 2500.0
