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


def _trace_share(rank, world, per_rank, n_pix):
    """The oracle standing in for one rank's GPU: trace the images bench.rank_images gives
    this rank (tiny cameras on the 64x32x32 torus)."""
    import math
    import numpy as np
    import bench
    import oracle as O
    from paper_2203_15963_gb300 import synth as S
    gp = S.GridParams(n_r=64, n_theta=32, n_phi=32)
    prims = {}
    out = []
    for k in bench.rank_images(rank, world, per_rank):
        spin, inc, phi = bench.image_spec(k, world)
        if spin not in prims:
            prims[spin] = S.make_torus(gp, spin, S.BASE_SEED)
        cam = S.Camera(theta=math.radians(inc), phi=phi, n=n_pix)
        r = O.trace(cam, S.Metric(spin=spin), gp, prims[spin], 230e9, nthreads=1)
        out.append((k, np.ascontiguousarray(r["stokes"]), np.ascontiguousarray(r["status"])))
    return out


def _shard_worker(rank, world, port, per_rank, n_pix, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = _trace_share(rank, world, per_rank, n_pix)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            out["gathered"] = [img for share in gathered for img in share]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_image_shares_union_equals_single_process():
    """Each rank traces its own share of the job's images (no collective on the data path);
    gathered in rank order, the shares are disjoint, cover every image once, and equal bit
    for bit what one process tracing the whole batch produces."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    world, per_rank, n_pix = 2, 3, 4
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_shard_worker, args=(world, port, per_rank, n_pix, out), nprocs=world,
                 join=True)
        got = list(out["gathered"])
    ks = [k for k, _, _ in got]
    assert ks == list(range(world * per_rank))
    shares = [set(bench.rank_images(r, world, per_rank)) for r in range(world)]
    assert not (shares[0] & shares[1])
    # the same images traced by one process (its own rank_images over the whole batch)
    single = [img for r in range(world) for img in _trace_share(r, world, per_rank, n_pix)]
    for (k1, s1, st1), (k2, s2, st2) in zip(got, single):
        assert k1 == k2
        assert np.array_equal(st1, st2)
        assert np.array_equal(s1, s2)
    # in the benchmark (9 images a rank) rank 1 sees the 9 spin/inclination pairs of rank 0
    # from the opposite azimuth
    import math
    assert bench.image_spec(9, 2)[:2] == bench.image_spec(0, 2)[:2]
    assert bench.image_spec(0, 2)[2] == 0.0 and bench.image_spec(9, 2)[2] == math.pi
