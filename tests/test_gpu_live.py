"""Live results (abp_live): every snapshot's moments and histogram rows reach the caller's
page-locked host buffers while the integration goes on.

Bars: bitwise equal to the histograms of the same run read at the end and to the moments
abp_reduce gives after integrating to the snapshot step in a separate run; every snapshot
arrives (more snapshots than the library keeps events for); pageable buffers and runs
without snapshots are refused.  Against the FP64 oracle run to each snapshot step (the
results the paper displays while a run goes on, Sec. 3.2): mean velocity within 3 standard
errors, histograms by a two-sample chi^2 test with p > 0.01.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1104_2499_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abp():
    from paper_1104_2499_gb300 import abp as A
    from paper_1104_2499_gb300 import build as B

    B.build()
    A.lib()
    return A


def live_batch(S=10, N=1000):
    sets = [W._with(D=0.1), W._with(D=0.3, F0=-0.2), W._with(D=0.05, asym=0.0)]
    sets += [W._with(D=0.02 * (i + 1), F0=0.01 * i) for i in range(40)]  # one-trajectory work items
    return W.Workload(name="live", sets=sets, n_traj=[600, 300, 5] + [1] * 40, n_steps=[N, N, N - 7] + [N] * 40,
                      dt=1e-3, seed=41, v0_mode=1, hist_x_bins=16, hist_v_bins=8, v_lo=-2.0, v_hi=2.0,
                      snapshot_every=S)


def pinned(shape, dtype):
    return torch.zeros(shape, dtype=dtype, pin_memory=True)


@pytest.mark.parametrize("schedule", [1, 2])
def test_live_snapshots_match_end_of_run_and_reduce(abp, schedule):
    w = live_batch()
    stream = torch.cuda.Stream()
    with abp.Ensemble(w, stream=stream, schedule=schedule, particles_per_thread=1) as ens:
        ens.set_params()
        ns = ens.n_snapshots()
        assert ns == 100  # more than the library's ring of in-flight snapshots
        S = len(w.sets)
        mom = pinned((ns, S, 8), torch.float64)
        hx = pinned((ns, S, w.hist_x_bins), torch.int32)
        hv = pinned((ns, S, w.hist_v_bins + 2), torch.int32)
        abp.abp_live(ens.ctx, mom, hx, hv)
        ens.integrate(-1)
        assert 0 <= abp.abp_live_ready(ens.ctx) <= ns
        ens.synchronize()
        assert abp.abp_live_ready(ens.ctx) == ns
        res = ens.results(host=True)
        assert torch.equal(hx, res["hist_x"]) and torch.equal(hv, res["hist_v"])
        # the last snapshot's moments are the end-of-run moments of the sets that ran to the end
        assert torch.equal(mom[-1], res["moments"])
    # moments at every 7th snapshot step against a run stopped at that step
    with abp.Ensemble(w, stream=stream, schedule=schedule, particles_per_thread=1) as ref:
        ref.set_params()
        done = 0
        for k in range(0, ns, 7):
            ref.integrate((k + 1) * w.snapshot_every - done)
            done = (k + 1) * w.snapshot_every
            r = ref.results(host=True)["moments"]
            assert torch.equal(mom[k], r), k


def test_live_restarts_after_reset_and_can_stop(abp):
    w = live_batch(S=100, N=600)
    stream = torch.cuda.Stream()
    with abp.Ensemble(w, stream=stream) as ens:
        ens.set_params()
        ns = ens.n_snapshots()
        mom = pinned((ns, len(w.sets), 8), torch.float64)
        abp.abp_live(ens.ctx, mom, None, None)
        ens.integrate(-1)
        ens.synchronize()
        first = mom.clone()
        mom.zero_()
        ens.reset()
        assert abp.abp_live_ready(ens.ctx) == 0
        ens.integrate(250)  # snapshots 0 and 1
        ens.synchronize()
        assert abp.abp_live_ready(ens.ctx) == 2
        assert torch.equal(mom[:2], first[:2]) and not mom[2:].any()
        abp.abp_live(ens.ctx, None, None, None)  # off: the rest is not sent
        ens.integrate(-1)
        ens.synchronize()
        assert not mom[2:].any()


def test_live_rejects_pageable_memory_and_missing_snapshots(abp):
    w = live_batch(S=100, N=300)
    with abp.Ensemble(w) as ens:
        ens.set_params()
        ns = ens.n_snapshots()
        pageable = torch.zeros((ns, len(w.sets), 8), dtype=torch.float64)
        with pytest.raises(abp.AbpError):
            abp.abp_live(ens.ctx, pageable, None, None)
        with pytest.raises(abp.AbpError):  # device memory is not a live destination either
            abp.abp_live(ens.ctx, torch.zeros((ns, len(w.sets), 8), dtype=torch.float64, device="cuda"), None, None)
    w0 = live_batch(S=100, N=300)
    w0.snapshot_every = 0
    with abp.Ensemble(w0) as ens:
        ens.set_params()
        with pytest.raises(abp.AbpError):
            abp.abp_live(ens.ctx, pinned((1, len(w0.sets), 8), torch.float64), None, None)


def _chi2_two_sample(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    if a.size < 2:
        return 1.0
    ka, kb = math.sqrt(b.sum() / a.sum()), math.sqrt(a.sum() / b.sum())
    return float(stats.chi2.sf(np.sum((ka * a - kb * b) ** 2 / (a + b)), a.size - 1))


def test_live_snapshots_match_the_oracle_at_each_snapshot_step(abp):
    # three sets of 1,200 to 3,000 trajectories, 1,900 or 2,000 steps, a snapshot every 500:
    # snapshot k must be the ensemble at step (k + 1) 500 of the oracle's run
    sets = [W._with(D=0.1), W._with(D=0.3, F0=-0.2, q=2.0), W._with(D=0.05, asym=0.0)]
    w = W.Workload(name="live_oracle", sets=sets, n_traj=[3000, 1200, 2500], n_steps=[2000, 2000, 1900], dt=1e-3,
                   seed=44, v0_mode=1, hist_x_bins=20, hist_v_bins=12, v_lo=-3.0, v_hi=3.0, snapshot_every=500)
    stream = torch.cuda.Stream()
    with abp.Ensemble(w, stream=stream) as ens:
        ens.set_params()
        ns = ens.n_snapshots()
        mom = pinned((ns, w.n_sets, 8), torch.float64)
        hx = pinned((ns, w.n_sets, w.hist_x_bins), torch.int32)
        hv = pinned((ns, w.n_sets, w.hist_v_bins + 2), torch.int32)
        abp.abp_live(ens.ctx, mom, hx, hv)
        ens.integrate(-1)
        ens.synchronize()
        assert abp.abp_live_ready(ens.ctx) == ns == 4
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        full = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                         v0_mode=w.v0_mode, snapshot_every=w.snapshot_every, hist_x_bins=w.hist_x_bins,
                         hist_v_bins=w.hist_v_bins, v_lo=w.v_lo, v_hi=w.v_hi)
        for k in range(ns):
            step = (k + 1) * w.snapshot_every
            if step > w.n_steps[i]:  # the set has ended: its rows stay at its last step's values
                assert int(hx[k, i].sum()) == 0
                continue
            r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=step, traj_base=base[i],
                          v0_mode=w.v0_mode)
            m = mom[k, i].numpy()
            assert abs(m[0] - r["mean_v"]) <= 3 * r["se_v"], (i, k, m[0], r["mean_v"], r["se_v"])
            assert m[1] == pytest.approx(r["se_v"], rel=0.1), (i, k)
            assert m[2] == pytest.approx(r["msd"], rel=0.1, abs=1e-6), (i, k)
            assert int(hx[k, i].sum()) == w.n_traj[i] and int(hv[k, i].sum()) == w.n_traj[i]
            assert _chi2_two_sample(hx[k, i].numpy(), full["hist_x"][k]) > 0.01, (i, k)
            assert _chi2_two_sample(hv[k, i].numpy(), full["hist_v"][k]) > 0.01, (i, k)
