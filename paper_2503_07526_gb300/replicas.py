"""Host-side logic of multi-GPU runs.

The path does not shard: every rank advances its own independent system (a
replica with its own seed) and no data crosses ranks during a run.  Ranks
meet only around the timed region, to agree on its duration (the slowest
rank) and to add up the work.  No collective runs inside a step.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's replica: distinct per rank, reproducible."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); the
    identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(atoms_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job atom-steps/s: every rank advanced atoms_per_rank atoms by
    steps steps; the job took the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("duration must be positive")
    return world * atoms_per_rank * steps / seconds
