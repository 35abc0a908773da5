"""Multi-GPU replicas of the solve.

The r starting points of a solve are independent (Section 4: each start runs its own copy of
Algorithm 2), so N GPUs each hold a replica of A and run their own share of the starts.  The
path needs no collective; after the solves one host-side exchange of two numbers per rank picks
the best start over all ranks (largest objective, ties to the lowest rank, as within a rank).
"""
from __future__ import annotations


def rank_starts(r_total: int, rank: int, world: int) -> tuple[int, int]:
    """(offset, count) of this rank's contiguous share of r_total starts."""
    if world < 1 or not 0 <= rank < world or r_total < 0:
        raise ValueError("bad rank/world/r")
    base, extra = divmod(r_total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def best_over_ranks(objective: float, world: int, dist=None) -> tuple[int, float]:
    """(winning rank, its objective) over all ranks; ties go to the lowest rank."""
    if world == 1 or dist is None:
        return 0, float(objective)
    import torch
    t = torch.tensor([float(objective)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    best = t.item()
    me = dist.get_rank()
    cand = torch.tensor([me if float(objective) == best else world], dtype=torch.int64)
    dist.all_reduce(cand, op=dist.ReduceOp.MIN)
    return int(cand.item()), best
