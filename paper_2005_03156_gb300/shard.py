"""Host-side sharding for runs on several GPUs (one process per GPU).

The join is data parallel over points (the paper runs independent point
shards per process, Sec. V): every rank holds a replica of the polygon set
and its own contiguous range of points, and no collective touches the data
path. The only collective is the timing reduction (max over ranks)."""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced [start, end) of n points for `rank` of `world`."""
    if world <= 0 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """All-reduce MAX of a scalar (e.g. a step time) over the process group;
    the value itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
