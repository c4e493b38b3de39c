"""Host logic of multi-GPU runs: independent replicas, no data-path collective.

The MSFV path does not shard: one process per GPU solves its own instance, with its own
seeded conductivity, sources and data.  The only communication is timing: a barrier
before the timed region and a MAX over ranks of the elapsed time, so the whole-job
throughput is (units all ranks processed) / (slowest rank's time).  These helpers are
backend-agnostic (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    rank: int
    world: int
    local: int


def rank_env(environ=None) -> RankEnv:
    """RANK / WORLD_SIZE / LOCAL_RANK as set by torch.distributed.run (defaults: one rank)."""
    env = os.environ if environ is None else environ
    return RankEnv(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")),
                   int(env.get("LOCAL_RANK", "0")))


@dataclass(frozen=True)
class ReplicaSeeds:
    model: int      # the conductivity the timed solves use
    truth: int      # the independent model that makes the observed data
    noise: int      # the 1% data noise


def replica_seeds(rank: int) -> ReplicaSeeds:
    """Seeds of rank `rank`'s instance: every replica solves a different problem."""
    if rank < 0:
        raise ValueError("rank must be >= 0")
    return ReplicaSeeds(model=2 + rank, truth=100 + rank, noise=7 + rank)


def max_over_ranks(value: float, device=None) -> float:
    """MAX of a per-rank float over the default process group (identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(world: int, units_per_rank: int, slowest_seconds: float) -> float:
    """Units per second of the whole job: every rank did units_per_rank units, and the job
    took as long as its slowest rank."""
    if world < 1 or units_per_rank < 0:
        raise ValueError("world >= 1 and units_per_rank >= 0 required")
    if slowest_seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return world * units_per_rank / slowest_seconds
