"""Index-range sharding across ranks (one process per GPU).

Every result of libvndf is a pure function of the inputs and of the global
sample index (Philox counter) or query index (Philox stream), so a batch is
split across ranks by giving each rank a contiguous range and the matching
counter base or stream base: no collective is needed on the data path.  The
only communication is the timing barrier and the max over ranks, plus, for a
fitting step split by texels, one sum of the per-shard loss shares (logging).
"""
import torch


def sample_shard(rank, world, n_per_rank):
    """(counter_base, n) of a rank's samples under weak scaling: global indices [rank n, (rank + 1) n)."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    return rank * int(n_per_rank), int(n_per_rank)


def query_shard(rank, world, n_queries):
    """(start, stop) of a rank's queries when n_queries are split as evenly as possible (strong scaling).

    The rank passes stream_id = start so that query q keeps the Philox stream it has in a single call.
    """
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    base, extra = divmod(int(n_queries), world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks (identity without an initialised process group)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def texel_shard(rank, world, n_texels):
    """(start, stop) of a rank's texels in a fitting step; the rank passes stream_id = start."""
    return query_shard(rank, world, n_texels)


def sum_over_ranks(value, device=None):
    """Sum of a float over all ranks in FP64 (identity without an initialised process group).

    A fitting step split by texels reports each shard's share of the loss (its texels'
    squared errors over the whole map's 3T components); their sum is the map's loss."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())
