"""The multi-process path of bench.py (replicas: one process per GPU, no
collective on the data path) on CPU with the gloo backend, world size 2:
the timing is the max over ranks and the throughput sums the ranks' work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    td.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    t = bench.reduce_max(1.0 + rank, w)          # rank 1 is the slow one
    cp = bench.reduce_sum(100.0 * (rank + 1), w)  # 100 + 200 CP iterations
    out[rank] = (t, cp, cp / t)
    td.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        t, cp, rate = out[rank]
        assert t == 2.0 and cp == 300.0 and rate == 150.0


def test_single_process_reductions_are_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(7.0, 1) == 7.0
