"""Live results (abp_live): every snapshot's moments and histogram rows reach the caller's
page-locked host buffers while the integration goes on.

Bars: bitwise equal to the histograms of the same run read at the end and to the moments
abp_reduce gives after integrating to the snapshot step in a separate run; every snapshot
arrives (more snapshots than the library keeps events for); pageable buffers and runs
without snapshots are refused.
"""
import numpy as np
import pytest

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
