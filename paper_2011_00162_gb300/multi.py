"""Host-side logic for runs on several ranks (one process per GPU).

The OD2P iteration of one reconstruction runs on one GPU.  Several GPUs run
independent work: replicas of one workload, or disjoint shares of a batch of
independent reconstructions.  Neither needs a data-path collective; the only
collective is the max-over-ranks of the timed interval.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(costs: list[float], rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` owns: greedy longest-processing-time
    assignment of the costs to `world` ranks (ties to the lowest rank), so every
    item has exactly one owner and the loads are balanced."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(value: float, device: torch.device | None = None) -> float:
    """Largest `value` over all ranks (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
