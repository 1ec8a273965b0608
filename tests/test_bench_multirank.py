"""The benchmark's multi-GPU path (independent replicas, weak scaling) with world size 2 on
the gloo backend: the timed region reduces to the slowest rank and the whole-job value counts
every rank's rays."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [0.8, 1.25][rank]                  # rank 1 is the slow one
        e = bench.reduce_elapsed(torch, elapsed, world, torch.device("cpu"))
        v = bench.weak_scaling_value(world, 9 * 65536, 5, e)
        out[rank] = (e, v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == pytest.approx(1.25) and res[1][0] == pytest.approx(1.25)
    assert res[0][1] == pytest.approx(2 * 9 * 65536 * 5 / 1.25)
    assert res[0] == res[1]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_elapsed(torch, 0.5, 1, torch.device("cpu")) == 0.5
    assert bench.weak_scaling_value(1, 100, 4, 2.0) == 200.0
