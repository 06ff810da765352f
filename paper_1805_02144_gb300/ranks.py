"""Rank bookkeeping of multi-GPU runs.

One trajectory of the method does not shard without a halo exchange per
J(u)x and an allreduce per IOM2 column; every rank therefore advances its own
replica of the workload (weak scaling) and nothing crosses ranks on the data
path.  Only timing does: each timed region is closed by a barrier and its
duration is the maximum over ranks, so the job's throughput is the units all
ranks processed divided by the slowest rank's time.  Independent ensemble
members split across ranks the same way (`member_shard`).
"""
from __future__ import annotations

import os
from dataclasses import dataclass
from typing import Mapping, Optional


@dataclass(frozen=True)
class Ranks:
    world: int
    rank: int
    local: int

    @property
    def lead(self) -> bool:
        """Rank 0 prints the job's result line."""
        return self.rank == 0


def from_env(env: Optional[Mapping[str, str]] = None) -> Ranks:
    """WORLD_SIZE / RANK / LOCAL_RANK as torchrun sets them (defaults: one rank)."""
    env = os.environ if env is None else env
    world = int(env.get("WORLD_SIZE", "1"))
    rank = int(env.get("RANK", "0"))
    local = int(env.get("LOCAL_RANK", str(rank)))
    if world < 1 or not 0 <= rank < world or local < 0:
        raise ValueError(f"inconsistent ranks: WORLD_SIZE={world} RANK={rank} LOCAL_RANK={local}")
    return Ranks(world, rank, local)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """max of x over the ranks of the default process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, t_ms: float) -> float:
    """Whole-job throughput (units/s): every rank's units over the slowest rank's time."""
    if world < 1 or units_per_rank < 0 or not t_ms > 0.0:
        raise ValueError("job_rate needs world >= 1, units >= 0 and a positive time")
    return world * units_per_rank / (t_ms / 1e3)


def member_shard(n_members: int, world: int, rank: int) -> range:
    """Contiguous block of ensemble members owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n_members < 0:
        raise ValueError("member_shard needs 0 <= rank < world and n_members >= 0")
    q, r = divmod(n_members, world)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))
