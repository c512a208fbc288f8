"""The multi-GPU path of bench.py runs independent replicas (the solve has no
data-parallel exchange): its only collective is the max over ranks of the
timed interval.  Checked here with two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [1.5, 2.5][rank]
    t_max = bench.max_over_ranks(t_local, world, "cpu")
    out[rank] = (t_max, bench.replica_value(409600, 10, t_max, world))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t_max, value = res[0]
    assert t_max == 2.5
    assert value == pytest.approx(2 * 409600 * 10 / 2.5)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_value(100, 4, 2.0, 1) == 200.0
