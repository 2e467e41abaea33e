"""Host-side logic of multi-GPU runs.  Problems are independent, so N GPUs solve N disjoint
shards with no collective on the data path; the only collectives are the timing barrier and
the max-over-ranks of the timed region (weak scaling: each rank has its own batch)."""
from __future__ import annotations


def shard(total: int, rank: int, world: int) -> range:
    """Contiguous block of problem indices of `rank` (sizes differ by at most one)."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def first_index(per_rank: int, rank: int) -> int:
    """First generator index of rank's own batch in a weak-scaling run."""
    return rank * per_rank


def max_over_ranks(values, dist=None, device=None):
    """Element-wise max of a list of floats over all ranks (identity without dist)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(values, dist=None, device=None):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()
