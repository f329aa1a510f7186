"""Multi-process (one process per GPU) helpers for the weak-scaling launch.

Instances are independent (the paper batches with map2 badd asss bsss,
Sec. V-A), so every rank runs its own batch with no collective on the data
path.  The only collectives are the timing barrier and a max-reduction of
the elapsed time over ranks.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic batch: disjoint streams per rank."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (identity without a process
    group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
