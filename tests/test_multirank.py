"""World-size-2 gloo test (CPU) of the replica aggregation bench.py uses for
N > 1: whole-job work is summed over ranks and time is the slowest rank's."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, w = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), world, torch.device("cpu"))
    q.put((rank, t, w))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, w in out:
        assert t == 2.0 and w == 30.0


def _shard_worker(rank, world, port, q):
    """Each rank computes its own target rows of the oracle matvec against all
    sources, then the rows are all-gathered (the exchange of a sharded run)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from oracle import mobility as om, rigid
    from paper_1709_02410_gb300 import synth
    from paper_1709_02410_gb300.partition import blob_ranges
    s = synth.boomerang_suspension(7, 6.0, 3)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    F = synth.gaussian(4, (3, s.n))
    prm = om.Params(synth.ETA, s.a)
    i0, i1 = blob_ranges(s.nb, s.nper, world)[rank]
    mine = om.apply(r, F, prm, rows=np.arange(i0, i1))
    parts = [None] * world
    dist.all_gather_object(parts, (i0, i1, mine))
    U = np.zeros((3, s.n))
    for a, b, u in parts:
        U[:, a:b] = u
    q.put((rank, float(np.abs(U - om.apply(r, F, prm)).max() / np.abs(U).max())))
    dist.destroy_process_group()


def test_row_sharded_matvec_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(180)
        assert p.exitcode == 0
    for rank, err in sorted(q.get(timeout=10) for _ in range(2)):
        assert err <= 1e-14


def test_body_ranges():
    from paper_1709_02410_gb300.partition import blob_ranges, body_ranges
    assert body_ranges(7, 2) == [(0, 4), (4, 7)]
    assert body_ranges(3, 4) == [(0, 1), (1, 2), (2, 3), (3, 3)]
    rr = blob_ranges(4369, 15, 8)
    assert rr[0][0] == 0 and rr[-1][1] == 65535
    assert all(b0 == a1 for (_, a1), (b0, _) in zip(rr, rr[1:]))
    assert max(b - a for a, b in rr) - min(b - a for a, b in rr) <= 15
