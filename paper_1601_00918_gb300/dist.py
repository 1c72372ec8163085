"""Multi-process helpers: one process per GPU, no collective on the data path.

The step of one grid is not split across GPUs; what shards is a sweep of
independent channels (each rank bisects its share) and, for the benchmark,
independent replicas (each rank steps its own copy).  The only collectives
are host-side: the maximum of the ranks' timings and the gather of the
ranks' results.  Works with NCCL (GPU tensors) and gloo (CPU tensors).
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (keeps uneven sizes mixed)."""
    return list(items)[rank::world]


def unshard(parts, n: int):
    """Inverse of shard: parts[r] holds the results of items r, r + world, ..."""
    world = len(parts)
    out = [None] * n
    for r, part in enumerate(parts):
        for k, v in enumerate(part):
            out[r + k * world] = v
    return out


def _device_for_backend():
    import torch
    import torch.distributed as dist
    return torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for_backend())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(local, n: int):
    """Results of a sharded list, back in the original order on every rank."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(local))
    return unshard(parts, n)
