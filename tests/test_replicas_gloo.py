"""The multi-rank bench path on CPU: two gloo ranks, each timing its own
replica; every rank must see the slowest rank's time and the whole-job
value must count every rank's node updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = 1.0 + rank  # rank 1 is slower
    tmax = bench.max_over_ranks(t, dist, torch.device("cpu"))
    val = bench.whole_job_glups(1000, 10, world, tmax)
    out[rank] = (tmax, val)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    # the manager process is spawned too: the oracle's OpenMP threads may
    # already run in this process, and a fork after them can deadlock
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    tmax, val = res[0]
    assert tmax == 2.0
    assert val == pytest.approx(1000 * 10 * 2 / 2.0 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_glups(16777216, 1000, 1, 0.175) == pytest.approx(95.87, rel=1e-3)
