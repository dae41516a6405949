"""Host logic of multi-process runs: one process per GPU, independent replicas.

The reconstruction of one volume is not split across GPUs (every GPU runs
whole reconstructions), so ranks split independent work items and the
only collective is the timing reduction (max over ranks).
"""


def shard(items, rank, world):
    """Round-robin share of `items` for `rank` (a partition over all ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(items)[rank::world]


def replica_seed(base, rank):
    """Seed of the synthetic volume that `rank` reconstructs."""
    return int(base) + int(rank)


def max_over_ranks(values, device=None):
    """Element-wise max of a list of floats over all ranks (no-op when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()
