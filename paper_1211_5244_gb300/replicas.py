"""Host logic of multi-GPU runs: independent replicas, one process per GPU.

The solve has no exchange step between GPUs (each density is a separate
problem), so N GPUs run N independent replicas: rank r solves its own
densities (seeded with seed + r), nothing crosses GPUs on the data path, and
the only collectives are a barrier around the timed region and one max-reduce
of the elapsed time, so that the reported throughput is the work of all ranks
divided by the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad torchrun environment: RANK={rank} WORLD_SIZE={world}")
    return rank, world, local


def replica_seed(seed, rank):
    """Seed of the density that rank `rank` solves."""
    return int(seed) + int(rank)


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value, dist, device="cpu"):
    """The maximum of a per-rank float over all ranks (the value itself without dist)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, seconds):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return world * units_per_rank / seconds


def aggregate(elapsed_s, units_per_rank, dist, device="cpu"):
    """(value, slowest elapsed seconds) for a timed region that ran on every rank."""
    world = dist.get_world_size() if dist is not None else 1
    slowest = max_over_ranks(elapsed_s, dist, device)
    return throughput(units_per_rank, world, slowest), slowest
