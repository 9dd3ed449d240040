"""Multi-rank host logic on CPU (gloo, world size 2): pose batches split across ranks,
each rank evaluates its share with the oracle, and the ranks agree on the argmax."""
import os
import socket

import numpy as np
import pytest

from paper_1709_06948_gb300 import shard


def test_shard_range_partitions():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_pack_argmax_order():
    keys = [shard.pack_argmax(m, i) for m, i in [(0.5, 3), (0.5, 1), (0.7, 9), (-1e-7, 0), (0.0, 2)]]
    assert shard.unpack_argmax(max(keys)) == 9
    assert shard.unpack_argmax(max(keys[:2])) == 1  # tie: lower index
    assert max(keys[3:]) == keys[4]                 # 0.0 > -1e-7


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    import scangen
    from tests.helpers import oracle_grid
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pair = scangen.tiny_pair()
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    etas = scangen.tiny_poses()
    lo, hi = shard.shard_range(len(etas), rank, world)
    mi, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(etas[lo:hi]))
    best = int(np.argmax(mi))  # numpy: first maximum = lowest index
    g = shard.global_argmax(float(np.float32(mi[best])), lo + best)
    t = shard.max_over_ranks(float(rank))
    out[rank] = (g, t)
    dist.destroy_process_group()


def test_two_rank_argmax_matches_single_process():
    import torch.multiprocessing as mp

    import oracle
    import scangen
    from tests.helpers import oracle_grid
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    pair = scangen.tiny_pair()
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    mi, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(scangen.tiny_poses()))
    expect = int(np.argmax(mi.astype(np.float32)))
    assert res[0][0] == res[1][0] == expect
    assert res[0][1] == res[1][1] == 1.0
