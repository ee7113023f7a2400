"""Bookkeeping of multi-GPU runs of one node.

The translation stage has no exchange step between directions, fields or
independent problems (Sec. II.C: restore and translation per direction need
no communication), so a run on N GPUs is N independent replicas, one process
per GPU: each rank translates its own problem, the only collectives are a
barrier around the timed region and the maximum of the per-rank times, and
the throughput counts the work of all ranks (weak scaling).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Ranks:
    world: int
    rank: int
    local: int

    @property
    def leader(self) -> bool:
        return self.rank == 0


def ranks_from_env(env=None) -> Ranks:
    """WORLD_SIZE / RANK / LOCAL_RANK as torchrun sets them (1 / 0 / 0 alone)."""
    env = os.environ if env is None else env
    world = int(env.get("WORLD_SIZE", "1"))
    rank = int(env.get("RANK", "0"))
    local = int(env.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"inconsistent ranks: WORLD_SIZE={world} RANK={rank}")
    return Ranks(world, rank, local)


def replica_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s problem: rank 0 keeps the workload's own seed."""
    return seed + 7919 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself alone)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second, timed by the slowest rank."""
    return world * units_per_rank / seconds
