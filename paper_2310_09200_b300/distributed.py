"""Several GPUs, one process each (torch.distributed; NCCL on GPUs, gloo on CPU).

Standard synthesis shards without exchange until the end: the images are a
plain sum over time steps (Algorithm 1), so each rank collects a contiguous
block of the steps into its own handle, and one sum-reduce of the
n_level x n_pix images gives the job's images. Independent jobs per rank
(weak scaling, as the benchmark runs them) need no collective at all beyond
the timing's max over ranks.
"""
from __future__ import annotations


def shard_steps(n_t: int, rank: int, world: int) -> range:
    """Contiguous block of the n_t steps for `rank`: the first n_t % world
    ranks take one step more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_t, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def sum_images(img, group=None):
    """Sum the ranks' partial images (a torch tensor, in place) and return it."""
    import torch.distributed as dist
    dist.all_reduce(img, op=dist.ReduceOp.SUM, group=group)
    return img


def max_over_ranks(value: float, device=None) -> float:
    """The largest of the ranks' values (the job ends when the slowest rank does)."""
    import torch
    import torch.distributed as dist
    x = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())
