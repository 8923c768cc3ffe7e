"""Process-level plumbing for running the operator on several GPUs of a node.

Cells are independent (the collision operator is local in x, Sec. 3.3), so the
work shards by cell with no exchange on the data path: each rank owns its
cells, and the only collectives are a barrier and the max of the per-rank
step time (for reporting).  One process per GPU, launched by torchrun.
"""
import os


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_cells, rank, world):
    """Contiguous cell range [begin, end) of `rank` when n_cells are split over
    `world` ranks as evenly as possible (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world) or n_cells < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_cells, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value, device=None):
    """Max of a float over all ranks of the default process group (identity
    when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
