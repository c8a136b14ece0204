"""The multi-GPU path of bench.py runs independent replicas (no data-path collective): the
job time is the max over ranks and the throughput sums the ranks' units.  Checked here with
two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_local = 1.0 + rank          # rank 1 is the slow one
    units = 100.0 * (rank + 1)    # units processed by this rank
    t, rate = bench.aggregate_ranks(dist, "cpu", t_local, units)
    out[rank] = (t, rate)
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, rate = out[r]
        assert t == 2.0                 # max over ranks
        assert rate == pytest.approx(300.0 / 2.0)


def test_single_process_aggregation_is_identity():
    import bench

    assert bench.aggregate_ranks(None, "cpu", 2.0, 10.0) == (2.0, 5.0)
