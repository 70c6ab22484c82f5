"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) with different
local times agree on the slowest rank's time, and the whole-job rate counts
the units of both ranks (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    dist.barrier()
    t = bench.max_over_ranks(local_ms)
    rate = bench.whole_job_rate(32, world, t / 1e3)
    out[rank] = (t, rate)
    dist.destroy_process_group()


def test_two_rank_max_time_and_rate():
    port = _free_port()
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 32 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
