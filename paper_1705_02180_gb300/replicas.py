"""Replica sharding across ranks (one process per GPU).

Trajectories are independent (Sec. "Self-Consistent Path Sampling": every rMD
trajectory starts from X_U on its own), so ranks take disjoint ranges of global
replica ids and share nothing on the data path. The noise of a replica is keyed by
its global id, so a sharded run gives the same trajectories as one process running
all replicas. The only collectives are for timing and reporting.
"""
from __future__ import annotations

import numpy as np


def replica_ids(rank: int, world: int, per_rank: int) -> np.ndarray:
    """Global replica ids of `rank` when every rank runs `per_rank` replicas."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("need 0 <= rank < world and per_rank >= 0")
    return np.arange(per_rank, dtype=np.int64) + rank * per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
