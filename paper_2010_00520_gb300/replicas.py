"""Bookkeeping of multi-GPU runs of one node.

The translation stage has no exchange step between directions, fields or
independent problems (Sec. II.C: restore and translation per direction need
no communication), so a run on N GPUs needs no data-path collective.  Two
ways to use N GPUs, one process each:
  * replicas (weak scaling): each rank translates its own problem;
  * direction shards (strong scaling): the ranks split the directions of one
    problem into contiguous blocks (`direction_block`) and each translates
    its block with a shard plan (FMMFFT_KEY_DIR_FIRST / _COUNT).
Either way the only collectives are a barrier around the timed region and the
maximum of the per-rank times.
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


def direction_block(n_dir: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of rank `rank`'s contiguous block of n_dir directions:
    sizes differ by at most one, larger blocks first, every direction once."""
    if world < 1 or not 0 <= rank < world or n_dir < world:
        raise ValueError(f"cannot split {n_dir} directions over {world} ranks")
    base, extra = divmod(n_dir, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


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
