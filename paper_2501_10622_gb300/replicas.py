"""Replica bookkeeping for multi-GPU runs.

The halo-finding path does not shard with a single exchange, so several GPUs
run independent replicas (one box per rank, no collective on the data path).
Only the timing is shared: every rank's step time is reduced with a max, and
the whole-job throughput is the particles of all ranks over that time.
"""
from __future__ import annotations

import os


def env_ranks():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank's box comes from its own seed."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(particles_per_rank: int, world: int, max_ms: float) -> float:
    """Mparticles/s of all ranks together, timed by the slowest rank."""
    return world * particles_per_rank / (max_ms / 1e3) / 1e6
