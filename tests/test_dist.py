"""World-size-2 gloo tests (CPU) of the multi-process host logic: sharding a
sweep's channels across ranks, gathering the results back in order, and the
job time as the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1601_00918_gb300 import dist as D


def test_shard_unshard_roundtrip():
    items = list(range(11))
    parts = [D.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert D.unshard(parts, len(items)) == items


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = [{"id": k, "lam": 32 + 16 * (k % 3)} for k in range(9)]
        mine = D.shard(specs, rank, world)
        # a stand-in for the per-rank bisection: a deterministic function of the spec
        local = [{"id": s["id"], "g": 1e-4 * (1 + s["id"]) * s["lam"] / 32} for s in mine]
        res = D.gather(local, len(specs))
        t = D.max_over_ranks(10.0 + rank)
        out[rank] = (res, t)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_gloo_sweep_sharding():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    expect = [{"id": k, "g": 1e-4 * (1 + k) * (32 + 16 * (k % 3)) / 32} for k in range(9)]
    for rank in range(world):
        res, t = out[rank]
        assert res == expect
        assert t == 11.0
