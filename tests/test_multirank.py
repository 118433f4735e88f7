"""The multi-GPU path of the benchmark, on CPU with two gloo ranks.

Renders are independent, so N GPUs run N replicas with rank-specific scenes
and no collective on the data path; the only exchange is the maximum of the
ranks' timings, which sets the job's time (weak scaling).  This checks that
exchange and the whole-job throughput, and that every rank renders a scene of
the same size but different content.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (mx, bench.job_throughput(world, 10, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_exchange_and_throughput():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    times = [12.5, 20.0]   # milliseconds for 10 renders on each rank
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, thr = res[r]
        assert mx == max(times)
        # 2 ranks x 10 renders in the slowest rank's 20 ms
        assert thr == pytest.approx(2 * 10 / 0.020)


def test_single_rank_needs_no_exchange():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 4, 2.0) == pytest.approx(2000.0)


def test_ranks_render_same_size_different_scenes():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.make_scene(0, n=2000, res=64)
    b = bench.make_scene(1, n=2000, res=64)
    assert a.pos.shape == b.pos.shape and (a.width, a.height) == (b.width, b.height)
    assert a.n_channels == b.n_channels and a.n_track == b.n_track
    assert not np.array_equal(a.pos, b.pos)
