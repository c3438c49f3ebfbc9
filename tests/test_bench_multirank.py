"""The multi-GPU path of bench.py is replicas: no data exchange, a barrier and a max-over-ranks
timing reduction. That host logic is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    # rank r pretends its 10 steps took 100*(r+1) ms in total and one end-to-end call (r+1) s
    res = bench.aggregate(100.0 * (rank + 1), 1.0 * (rank + 1), 10, world, dist, "cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_per_step, value, e2e = res[r]
        assert ms_per_step == pytest.approx(20.0)          # slowest rank: 200 ms over 10 steps
        assert value == pytest.approx(world * 10 / 0.2)    # all ranks' units over the slowest time
        assert e2e == pytest.approx(world / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate(50.0, 0.5, 5, 1) == (10.0, 100.0, 2.0)
