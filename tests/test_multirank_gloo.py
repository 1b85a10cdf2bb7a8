"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank gets its own problem
(weak scaling, no collective on the data path) and the job throughput uses the slowest rank's time."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 1000.0 + 500.0 * rank          # rank 1 is the slower one
        value, total = bench.aggregate(local_ms, steps=4, world=world, dist=dist, device="cpu")
        out[rank] = (value, total, bench.rank_seed(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_aggregate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        value, total, seed = res[rank]
        assert total == pytest.approx(1500.0)                  # MAX over ranks
        assert value == pytest.approx(world * 4 / 1.5)          # all ranks' solves / slowest time
    assert res[0][2] != res[1][2]                              # independent problems per rank


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, total = bench.aggregate(250.0, steps=5, world=1)
    assert total == 250.0 and value == pytest.approx(20.0)
