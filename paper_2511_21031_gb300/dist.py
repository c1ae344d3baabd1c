"""Host-side logic of the multi-GPU form.

Cells are independent during the bubble source update (every (cell, bin) has a
single owner and no exchange), so N GPUs run N independent blocks of cells:
weak scaling with no collective on the data path.  The only collectives are
the timing barrier and the max over ranks of the timed region.
"""
from __future__ import annotations

import os


def env_rank():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's own block of cells: every rank draws different phases."""
    return int(base_seed) + 1000 * int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over the default process group (the value itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, ms_max: float, world_size: int) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    if ms_max <= 0:
        raise ValueError("timed region must be positive")
    return units_per_rank * world_size / (ms_max * 1e-3)
