"""Replica sharding across GPUs.

The replicas of a workload are independent chains, so N GPUs partition them
with no exchange on the data path: rank r anneals its own block of global
replica indices (its random streams are those replicas' streams), and the only
collective is the final reduction of the best energy (and, in the benchmark,
of the step time).  Two modes:

  weak   -- every rank anneals `replicas` chains; rank r owns global indices
            [r*replicas, (r+1)*replicas).
  strong -- `replicas` chains in total, split as evenly as possible.
"""
from __future__ import annotations


def replica_range(rank: int, world: int, replicas: int, mode: str = "weak") -> tuple[int, int]:
    """-> (first global replica index, count) owned by `rank`."""
    if world < 1 or not 0 <= rank < world or replicas < 0:
        raise ValueError("bad rank/world/replicas")
    if mode == "weak":
        return rank * replicas, replicas
    if mode == "strong":
        base, extra = divmod(replicas, world)
        first = rank * base + min(rank, extra)
        return first, base + (1 if rank < extra else 0)
    raise ValueError(mode)


def reduce_best(local_best, group=None):
    """All-reduce (min) of this rank's best energy over the group (torch.distributed)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(local_best)], dtype=torch.int64)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return int(t.item())
