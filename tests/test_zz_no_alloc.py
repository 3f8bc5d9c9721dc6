"""The allocation-free entry point (abp_run_set_noalloc) against the context entry points.

Callers that cannot allocate device memory (a host framework that owns all device memory
through its own pool, a loop that must not stall on cudaMalloc) use abp_run_set_noalloc,
whose scratch is a static device array.  It must give the same moments and histograms as
abp_set_params + abp_integrate + abp_reduce for the same set, on consecutive calls that
reuse the shared scratch.  Collected last on purpose (file name) so that a failure here
does not hide the other tests in a run that stops at the first failure.
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


def _reference(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res = ens.results()
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in res.items()}


def _noalloc(A, w, **kw):
    cfg = A.make_config(w, **kw)
    ns = A.noalloc_snapshots(cfg, w.n_steps[0])
    mom = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    hx = torch.full((max(ns, 1), max(w.hist_x_bins, 1)), -1, dtype=torch.int32, device="cuda")
    hv = torch.full((max(ns, 1), w.hist_v_bins + 2), -1, dtype=torch.int32, device="cuda")
    A.abp_run_set_noalloc(w.sets[0], cfg, w.n_traj[0], w.n_steps[0], mom, hx if w.hist_x_bins else None,
                          hv if w.hist_v_bins else None)
    torch.cuda.synchronize()
    return mom, hx, hv


def test_noalloc_matches_context_entry_points_on_consecutive_calls(abp):
    cases = [
        W.Workload(name="na1", sets=[W._with(D=0.1)], n_traj=[3001], n_steps=[1500], dt=1e-3, seed=41, v0_mode=1,
                   hist_x_bins=64, hist_v_bins=30, v_lo=-3.0, v_hi=3.0, snapshot_every=500),
        W.Workload(name="na2", sets=[W._with(D=0.4, q=2.5, asym=0.1)], n_traj=[777], n_steps=[1203], dt=1e-3,
                   seed=42, v0_mode=0, hist_x_bins=32, hist_v_bins=10, v_lo=-2.0, v_hi=2.0, snapshot_every=400),
    ]
    for w in cases:  # two calls in a row share (and reuse) the static scratch
        ref = _reference(abp, w)
        mom, hx, hv = _noalloc(abp, w)
        # same kernels, same arithmetic: agreement far inside the 3-SE / 1e-4 bars of the
        # oracle comparisons; the histograms are integer counts and must be equal
        np.testing.assert_allclose(mom.cpu().numpy(), ref["moments"][0].cpu().numpy(), rtol=1e-12, atol=1e-15)
        assert torch.equal(hx, ref["hist_x"][:, 0, :])
        assert torch.equal(hv, ref["hist_v"][:, 0, :])
        assert int(hx[0].sum()) == w.n_traj[0]


def _case(n_traj, n_steps, seed, **kw):
    return W.Workload(name="na", sets=[W._with(D=0.2, q=1.5, asym=0.2)], n_traj=[n_traj], n_steps=[n_steps], dt=1e-3,
                      seed=seed, v0_mode=1, hist_x_bins=24, hist_v_bins=12, v_lo=-3.0, v_hi=3.0, snapshot_every=250,
                      **kw)


@pytest.mark.parametrize("n_traj,ppt,spl,scheme", [
    (2049, 1, 0, 0), (2049, 2, 0, 0), (2049, 4, 0, 0),  # trajectories per thread: tile sizes 256, 512, 1024
    (1500, 2, 333, 0),                                  # launches of 333 steps: 1,000 is no multiple of it
    (1500, 2, 0, 1),                                    # stochastic Heun
    (65536, 4, 0, 0),                                   # the capacity of the static scratch, all of it
    (65536, 1, 0, 0),                                   # ... with the largest tile table
])
def test_noalloc_configurations_bitwise_against_the_context(abp, n_traj, ppt, spl, scheme):
    # The context runs the same tiles (256 x particles_per_thread trajectories each) in the
    # lockstep schedule, so states, histograms and the fixed-order FP64 sums -- and with them
    # every moment -- must be the same bits, on two consecutive calls of the entry point.
    w = _case(n_traj, 1000, seed=43 + ppt, scheme=scheme)
    ref = _reference(abp, w, particles_per_thread=ppt, schedule=1, steps_per_launch=spl)
    for _ in range(2):
        mom, hx, hv = _noalloc(abp, w, particles_per_thread=ppt, schedule=1, steps_per_launch=spl)
        assert torch.equal(mom, ref["moments"][0]), (mom.cpu().numpy(), ref["moments"][0].cpu().numpy())
        assert torch.equal(hx, ref["hist_x"][:, 0, :])
        assert torch.equal(hv, ref["hist_v"][:, 0, :])


def test_noalloc_empty_ensemble_and_zero_steps(abp):
    # no trajectory: all moments zero, histograms cleared (after a call that filled them)
    _noalloc(abp, _case(300, 500, seed=50))
    mom, hx, hv = _noalloc(abp, _case(0, 500, seed=50))
    assert torch.count_nonzero(mom) == 0
    assert int(hx.sum()) == 0 and int(hv.sum()) == 0
    # no step: the time average is 0; the one final snapshot holds the initial condition
    w = _case(300, 0, seed=51)
    w.snapshot_every = 0
    mom, hx, hv = _noalloc(abp, w)
    assert float(mom[0]) == 0.0 and float(mom[2]) == 0.0 and int(hx[0].sum()) == 300


def test_noalloc_rejects_what_it_cannot_run(abp):
    w = W.single_set(n_traj=10, n_steps=10)
    cfg = abp.make_config(w)
    mom = torch.empty(8, dtype=torch.float64, device="cuda")
    hx = torch.empty((1, w.hist_x_bins), dtype=torch.int32, device="cuda")
    with pytest.raises(abp.AbpError) as ei:
        abp.abp_run_set_noalloc(w.sets[0], cfg, 65537, 10, mom, hx)
    assert ei.value.status == abp.ABP_EINVAL and "65536" in str(ei.value)
    # the work queue is not run by this entry point: refused, not ignored
    cfg2 = abp.make_config(w, schedule=2)
    with pytest.raises(abp.AbpError) as ei:
        abp.abp_run_set_noalloc(w.sets[0], cfg2, 10, 10, mom, hx)
    assert ei.value.status == abp.ABP_EINVAL and "lockstep" in str(ei.value)
    # the C side refuses host memory for outputs its kernels write (called past the wrapper)
    import ctypes as C

    host_mom = torch.empty(8, dtype=torch.float64, pin_memory=True)
    p = abp.abp_params()
    for k in W.PARAM_NAMES:
        setattr(p, k, float(w.sets[0][k]))
    err = C.create_string_buffer(256)
    st = abp.lib().abp_run_set_noalloc(C.byref(p), C.byref(cfg), 10, 10, host_mom.data_ptr(), hx.data_ptr(), None,
                                       None, err, 256)
    assert st == abp.ABP_EINVAL and b"current device" in err.value
