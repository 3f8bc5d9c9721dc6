"""Running one ensemble on several processes (one GPU each) and combining the results.

Trajectories and parameter sets are independent, and the noise of a trajectory is keyed by
its global id, so a batch shards with no exchange on the data path: each rank integrates its
trajectories (``abp_config.traj_base`` = the global id of its first one) and only the four
per-set sums of the ensemble reduction -- sum vbar, sum vbar^2, sum dx, sum dx^2 -- are
added across ranks at the end.  The moments of the combined ensemble are then formed by the
library (``abp_combine_moments``), with the formulas of its own reduction; nothing here
computes them.
"""
from __future__ import annotations

import numpy as np

from . import abp as A


def replica_traj_base(rank: int, total_traj: int) -> int:
    """Weak scaling: rank r integrates its own copy of the batch, trajectories
    [r T, (r + 1) T) of a larger ensemble (T = trajectories of one copy)."""
    return int(rank) * int(total_traj)


def combine(local_moments, n_traj_per_rank, n_steps, dt: float, world: int, all_reduce) -> np.ndarray:
    """Add the local per-set sums (columns 4..7 of abp_reduce's [n_sets, 8] moments) over
    ``world`` ranks with ``all_reduce`` (a callable summing a float64 array across ranks and
    returning it, e.g. around torch.distributed) and return the [n_sets, 8] moments of the
    combined ensemble of world x n_traj_per_rank[s] trajectories per set (host array)."""
    local = np.asarray(local_moments, dtype=np.float64)
    sums = all_reduce(np.ascontiguousarray(local[:, 4:8]))
    out = np.zeros((local.shape[0], 8))
    out[:, 4:8] = sums
    A.abp_combine_moments(out, [int(m) * world for m in n_traj_per_rank], list(n_steps), dt)
    return out


def all_reduce_sums_(moments, all_reduce, n_traj_total, n_steps, dt: float, stream=None) -> None:
    """In place on a torch moments tensor [n_sets, 8] (host or device): add the per-set sums
    (columns 4..7) across ranks, then recompute columns 0..3 for the combined ensemble of
    n_traj_total[s] trajectories per set.  The columns are a strided view, which collectives
    do not take, so they are reduced through a contiguous copy and written back."""
    sums = moments[:, 4:8].contiguous()
    all_reduce(sums)
    moments[:, 4:8].copy_(sums)
    A.abp_combine_moments(moments, n_traj_total, n_steps, dt, stream)
