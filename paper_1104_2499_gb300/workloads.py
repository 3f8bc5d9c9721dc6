"""Seeded synthetic workloads shaped like the paper's parameter sweeps.

This module only builds inputs (parameter sets, ensemble sizes, step counts, seeds); it
holds none of the method's arithmetic, so both the CUDA path and the FP64 oracle can use
it.  The paper (Sec. 2) sweeps one parameter per work item and averages over noise
realisations; it prints no default values for the model parameters, so the defaults below
are a reading: q = 1, c = 0.1, d = 1, gamma0 = 1, F0 = 0, h = 1, L = 1, a = 1/4 (the
weight printed in Eq. (pot)).  With them q d / c > gamma0, i.e. the depot drives active
motion with |v| -> sqrt(q/gamma0 - c/d).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PARAM_NAMES = ("q", "c", "d", "gamma0", "F0", "D", "h", "L", "asym")

DEFAULTS = dict(q=1.0, c=0.1, d=1.0, gamma0=1.0, F0=0.0, D=0.1, h=1.0, L=1.0, asym=0.25)


@dataclass
class Workload:
    """A batch of parameter sets integrated together.

    ``sets`` is a list of parameter dicts; ``n_traj[i]`` trajectories of set i run
    ``n_steps[i]`` Euler-Maruyama steps.  Trajectory ids are global: set i owns ids
    ``[sum(n_traj[:i]), sum(n_traj[:i+1]))``.
    """

    name: str
    sets: list
    n_traj: list
    n_steps: list
    dt: float = 1e-3
    seed: int = 0
    v0_mode: int = 0            # 0: v0 = 0; 1: v0 ~ N(0, sqrt(D))
    hist_x_bins: int = 0
    hist_v_bins: int = 0
    v_lo: float = -5.0
    v_hi: float = 5.0
    snapshot_every: int = 0     # 0: one snapshot after the last step
    checkpoint_every: int = 0
    scheme: int = 0             # 0: Euler-Maruyama (the paper's step), 1: stochastic Heun
    noise: int = 0              # 0: counter-based Philox, 1: xorshift per trajectory (Fig. 1)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_sets(self) -> int:
        return len(self.sets)

    @property
    def total_traj(self) -> int:
        return int(sum(self.n_traj))

    @property
    def particle_steps(self) -> int:
        return int(sum(int(m) * int(n) for m, n in zip(self.n_traj, self.n_steps)))

    def traj_base(self) -> list:
        out, acc = [], 0
        for m in self.n_traj:
            out.append(acc)
            acc += int(m)
        return out

    def param_matrix(self) -> np.ndarray:
        """[n_sets, 9] float64 in PARAM_NAMES order."""
        return np.array([[float(s[k]) for k in PARAM_NAMES] for s in self.sets], dtype=np.float64)


def params(**kw) -> dict:
    """One parameter set: the defaults (q, c, d, gamma0, F0, D, h, L, asym) with the given
    overrides."""
    p = dict(DEFAULTS)
    p.update(kw)
    return p


_with = params


def single_set(n_traj=4096, n_steps=10_000, D=0.1, seed=0, hist_x_bins=256, **kw) -> Workload:
    """One parameter set: 4,096 trajectories x 10^4 steps, dt = 1e-3, D = 0.1, x0 ~ U[0, L),
    v0 = e0 = 0, Philox seed 0; outputs <v> and a 256-bin histogram of x mod L."""
    return Workload(name="single_set_4096x1e4", sets=[_with(D=D, **kw)], n_traj=[n_traj],
                    n_steps=[n_steps], dt=1e-3, seed=seed, v0_mode=0, hist_x_bins=hist_x_bins)


def sweep_grid(n_D=64, n_q=32, traj_per_set=1024, n_steps=100_000, seed=1, hist_x_bins=256) -> Workload:
    """64 x 32 grid: D log-spaced in [1e-3, 1], q log-spaced in [0.1, 10], 1,024 trajectories
    per point (2,097,152 in all) x 10^5 steps, dt = 1e-3, v0 ~ N(0, sqrt(D)), Philox seed 1.
    Set index = iD * n_q + iq."""
    Ds = np.logspace(-3, 0, n_D)
    qs = np.logspace(-1, 1, n_q)
    sets = [_with(D=float(D), q=float(q)) for D in Ds for q in qs]
    n = len(sets)
    return Workload(name="sweep_D%dxq%d_%dtraj_%dsteps" % (n_D, n_q, traj_per_set, n_steps), sets=sets,
                    n_traj=[traj_per_set] * n, n_steps=[n_steps] * n, dt=1e-3, seed=seed, v0_mode=1,
                    hist_x_bins=hist_x_bins)


def uneven_batch(n_sets=512, seed=2, m_range=(256, 65_536), n_range=(10_000, 1_000_000)) -> Workload:
    """512 sets: D log-uniform in [1e-3, 1], asymmetry uniform in [0, 0.5], ensemble size
    log-uniform in [256, 65536], step count log-uniform in [1e4, 1e6]; dt = 1e-3, seed 2.
    The set parameters come from numpy's seeded generator (input construction only)."""
    rng = np.random.default_rng(seed)
    D = np.exp(rng.uniform(math.log(1e-3), math.log(1.0), n_sets))
    a = rng.uniform(0.0, 0.5, n_sets)
    M = np.rint(np.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1]), n_sets))).astype(np.int64)
    N = np.rint(np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), n_sets))).astype(np.int64)
    sets = [_with(D=float(D[i]), asym=float(a[i])) for i in range(n_sets)]
    return Workload(name="uneven_%dsets" % n_sets, sets=sets, n_traj=[int(m) for m in M],
                    n_steps=[int(n) for n in N], dt=1e-3, seed=seed, v0_mode=0, hist_x_bins=256)


def differentiation(n_traj=1 << 20, n_steps=100_000, seed=3, checkpoint_every=1000) -> Workload:
    """1M trajectories x 10^5 steps, D = 0.05, gradient of <v> w.r.t. (D, q, c, d, gamma0, a),
    checkpoints every 1,000 steps; seed 3."""
    return Workload(name="grad_%dx%d" % (n_traj, n_steps), sets=[_with(D=0.05)], n_traj=[n_traj],
                    n_steps=[n_steps], dt=1e-3, seed=seed, v0_mode=0, checkpoint_every=checkpoint_every)


def large_snapshots(n_traj=1 << 26, n_steps=1_000_000, seed=4, snapshot_every=10_000, bins=1024) -> Workload:
    """64M trajectories x 10^6 steps, D = 0.2, histograms of x mod L (1,024 bins) and of v in
    [-5, 5) (1,024 bins) every 10^4 steps; seed 4."""
    return Workload(name="snapshots_%dx%d" % (n_traj, n_steps), sets=[_with(D=0.2)], n_traj=[n_traj],
                    n_steps=[n_steps], dt=1e-3, seed=seed, v0_mode=0, hist_x_bins=bins, hist_v_bins=bins,
                    v_lo=-5.0, v_hi=5.0, snapshot_every=snapshot_every)


def force_sweep(n_F=64, F_lo=-1.0, F_hi=1.0, traj_per_set=4096, n_steps=100_000, D=0.1, seed=6) -> Workload:
    """The paper's benchmark observable, Fig. 2 and Sec. 2: mean velocity against the external
    (opposing) force F0, one parameter set per force value, n_F values evenly spaced in
    [F_lo, F_hi], the other parameters at their defaults."""
    Fs = np.linspace(F_lo, F_hi, n_F)
    sets = [_with(D=D, F0=float(F)) for F in Fs]
    return Workload(name="force_sweep_%dx%d_%dsteps" % (n_F, traj_per_set, n_steps), sets=sets,
                    n_traj=[traj_per_set] * n_F, n_steps=[n_steps] * n_F, dt=1e-3, seed=seed, v0_mode=0)


def shrink(w: Workload, max_traj: int | None = None, max_steps: int | None = None, max_sets: int | None = None,
           name: str | None = None) -> Workload:
    """A smaller copy of a workload (same parameter values) for parity runs."""
    sets, M, N = list(w.sets), list(w.n_traj), list(w.n_steps)
    if max_sets is not None and len(sets) > max_sets:
        idx = np.linspace(0, len(sets) - 1, max_sets).round().astype(int)
        sets = [sets[i] for i in idx]
        M = [M[i] for i in idx]
        N = [N[i] for i in idx]
    if max_traj is not None:
        M = [min(int(m), max_traj) for m in M]
    if max_steps is not None:
        N = [min(int(n), max_steps) for n in N]
    return replace(w, name=name or (w.name + "_small"), sets=sets, n_traj=M, n_steps=N)
