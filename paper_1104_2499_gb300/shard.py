"""Running one ensemble on several processes (one GPU each) and combining the results.

Trajectories and parameter sets are independent, and the noise of a trajectory is keyed by
its global id, so a batch shards with no exchange on the data path: each rank integrates its
trajectories (``abp_config.traj_base`` = the global id of its first one) and only the four
per-set sums of the ensemble reduction -- sum vbar, sum vbar^2, sum dx, sum dx^2 -- are
added across ranks at the end, after which the moments follow as for a single process.
"""
from __future__ import annotations

import numpy as np


def replica_traj_base(rank: int, total_traj: int) -> int:
    """Weak scaling: rank r integrates its own copy of the batch, trajectories
    [r T, (r + 1) T) of a larger ensemble (T = trajectories of one copy)."""
    return int(rank) * int(total_traj)


def moments_from_sums(sums, n_traj, n_steps, dt: float) -> np.ndarray:
    """[n_sets, 8] moments (mean_v, se_v, msd, d_eff, then the four sums) from the
    per-set sums [n_sets, 4] of M_s trajectories of N_s steps each -- the same formulas
    as the device reduction."""
    sums = np.asarray(sums, dtype=np.float64).reshape(-1, 4)
    M = np.asarray(n_traj, dtype=np.float64).reshape(-1)
    N = np.asarray(n_steps, dtype=np.float64).reshape(-1)
    out = np.zeros((sums.shape[0], 8))
    out[:, 4:] = sums
    with np.errstate(divide="ignore", invalid="ignore"):
        mean_v = np.where(M > 0, sums[:, 0] / M, 0.0)
        var_v = np.where(M > 1, (sums[:, 1] - M * mean_v * mean_v) / (M - 1), 0.0)
        msd = np.where(M > 0, sums[:, 3] / M, 0.0)
        mdx = np.where(M > 0, sums[:, 2] / M, 0.0)
        T = N * dt
        out[:, 0] = mean_v
        out[:, 1] = np.where(M > 0, np.sqrt(np.maximum(var_v, 0.0) / np.where(M > 0, M, 1)), 0.0)
        out[:, 2] = msd
        out[:, 3] = np.where(T > 0, (msd - mdx * mdx) / (2 * np.where(T > 0, T, 1)), 0.0)
    return out


def combine(local_moments, n_traj_per_rank, n_steps, dt: float, world: int, all_reduce) -> np.ndarray:
    """Add the local per-set sums over ``world`` ranks with ``all_reduce`` (a callable
    summing a float64 array in place across ranks, e.g. torch.distributed) and return the
    moments of the combined ensemble."""
    sums = np.ascontiguousarray(np.asarray(local_moments, dtype=np.float64)[:, 4:8])
    sums = all_reduce(sums)
    M = np.asarray(n_traj_per_rank, dtype=np.float64) * world
    return moments_from_sums(sums, M, n_steps, dt)


def all_reduce_sums_(moments, all_reduce) -> None:
    """In place: add the per-set sums (columns 4..7) of a torch moments tensor [n_sets, 8]
    across ranks.  The columns are a strided view, which collectives do not take, so they
    are reduced through a contiguous copy and written back."""
    sums = moments[:, 4:8].contiguous()
    all_reduce(sums)
    moments[:, 4:8].copy_(sums)
