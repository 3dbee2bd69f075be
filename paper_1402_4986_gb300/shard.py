"""Query sharding over several GPUs: one process per GPU, data replicated.

Each rank interpolates a contiguous slice of the queries against the full
data set.  Eq. 1 is independent per query, so no collective touches the
data path; the only communication is the optional gather of the results
and the max-over-ranks timing used by the benchmark.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def query_range(m: int, world: int, rank: int):
    """Contiguous [lo, hi) slice of m queries for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or m < 0:
        raise ValueError("bad shard arguments")
    return m * rank // world, m * (rank + 1) // world


def interpolate_sharded(data, queries, p: float = 2.0, group=None, gather: bool = True,
                        interpolate_fn=None):
    """Interpolate this rank's slice of `queries`; optionally all-gather Z.

    ``interpolate_fn(data, queries, p)`` defaults to the CUDA forward pass.
    Every rank must call this with the same data and queries.
    """
    if interpolate_fn is None:
        from . import interpolate as interpolate_fn
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    m = queries.shape[0]
    lo, hi = query_range(m, world, rank)
    local = interpolate_fn(data, queries[lo:hi].contiguous(), p)
    if not gather:
        return local
    width = (m + world - 1) // world
    padded = torch.zeros(width, dtype=local.dtype, device=local.device)
    padded[: hi - lo] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([parts[r][: query_range(m, world, r)[1] - query_range(m, world, r)[0]]
                      for r in range(world)])


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest `value` over all ranks (the benchmark's timing rule)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
