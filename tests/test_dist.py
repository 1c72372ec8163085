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


def _sweep_worker(rank, world, port, out):
    """One rank of sweep.run_sweep_sharded with the per-rank bisection
    replaced by a stub that echoes which channel and which bracket it was
    handed, so the test sees the library's own split of specs and brackets
    and its gather back into order."""
    import time

    import numpy as np
    import torch.distributed as dist

    from paper_1601_00918_gb300 import sweep
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def stub(lbm, specs, lo, hi, **kw):
        assert lbm == "lib" and kw == {"precision": "fp32"}
        time.sleep(0.01)
        return [{"lam": s.lam, "theta": s.theta_deg, "g_lo": float(a), "g_hi": float(b), "rank": rank}
                for s, a, b in zip(specs, lo, hi)], 1.0 + rank

    sweep.run_sweep = stub
    try:
        from paper_1601_00918_gb300 import workloads as wl
        specs = wl.sweep_specs(7, seed=3, lambdas=(32, 48, 64))
        lo = np.array([1e-5 * (k + 1) for k in range(7)])
        hi = 3.0 * lo
        res, dt = sweep.run_sweep_sharded("lib", specs, lo, hi, precision="fp32")
        out[rank] = ([(r["lam"], r["theta"], r["g_lo"], r["g_hi"], r["rank"]) for r in res], dt,
                     [(s.lam, s.theta_deg) for s in specs])
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_sharded_sweep_pairs_brackets_with_channels():
    """sweep.run_sweep_sharded on two gloo ranks: every channel is bisected
    by exactly one rank (round-robin), with its own bracket (not a
    neighbour's), the gathered results come back in the specs' order on both
    ranks, and the job time is the slower rank's."""
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_sweep_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        res, dt, specs = out[rank]
        assert dt == 2.0
        assert len(res) == 7
        for k, (lam, theta, g_lo, g_hi, who) in enumerate(res):
            assert (lam, theta) == specs[k]
            assert g_lo == 1e-5 * (k + 1) and g_hi == 3.0 * g_lo
            assert who == k % world
    assert out[0][0] == out[1][0]
