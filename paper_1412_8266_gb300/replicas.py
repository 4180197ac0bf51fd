"""Replica placement for runs on several GPUs (one process per GPU).

The path has no exchange step: every stream is independent (paper Sec. 2.1,
one stream per processing element).  Running on N GPUs is therefore N
replicas of the same workload on disjoint stream ranges of one stream set --
rank r owns streams [r S, (r+1) S) -- with no collective on the data path.
Only the timing is combined: the job's time is the slowest rank's time.
"""
from __future__ import annotations


def stream_range(rank: int, world: int, per_rank: int):
    """(first stream, count) owned by `rank` of `world` replicas."""
    if not 0 <= rank < world or per_rank <= 0:
        raise ValueError("need 0 <= rank < world and per_rank > 0")
    return rank * per_rank, per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (identity
    when torch.distributed is not initialised or has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
