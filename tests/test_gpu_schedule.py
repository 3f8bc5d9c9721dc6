"""Work-queue schedule (persistent launch over (tile, round) items), CUDA-graph replay of
repeated windows, the autotuner's choices and failure detection by a bounded wait.

Bars: the work-queue schedule, the lockstep schedule and graph replays give bitwise the
same state and results; the uneven batch agrees with the FP64 oracle within 3 SE; an
injected missing completion ends the launch with ABP_ETIMEOUT and leaves the context usable.
"""
import os
import time

import numpy as np
import pytest

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


def uneven(n_sets=24, seed=2):
    # the uneven-batch shape at test size: ensemble sizes log-uniform in [256, 4096], step
    # counts log-uniform in [500, 12000], asymmetry uniform in [0, 0.5]
    return W.uneven_batch(n_sets=n_sets, seed=seed, m_range=(256, 4096), n_range=(500, 12_000))


def run(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res = ens.results()
        st = ens.state()
        torch.cuda.synchronize()
        return res, st, ens.tuning()


@pytest.mark.parametrize("ppt", [1, 2])
def test_work_queue_matches_lockstep_bitwise(abp, ppt):
    w = uneven()
    w.hist_x_bins, w.hist_v_bins, w.snapshot_every = 32, 16, 700
    ra, sa, ta = run(abp, w, schedule=2, steps_per_launch=1000, particles_per_thread=ppt)
    rb, sb, tb = run(abp, w, schedule=1, steps_per_launch=4096, particles_per_thread=ppt)
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k
    assert ta["schedule"] == 2 and ta["steps_per_item"] == 1000 and ta["blocks"] > 0
    assert tb["schedule"] == 1 and tb["steps_per_item"] == 4096


def test_uneven_batch_against_oracle(abp):
    w = uneven()
    res, _, _ = run(abp, w)
    mom = res["moments"].cpu().numpy()
    base = w.traj_base()
    for i in (0, 5, 11, 17, 23):
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, hist_x_bins=w.hist_x_bins)
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * r["se_v"], i
        assert np.all(res["hist_x"].cpu().numpy()[0, i].sum() == w.n_traj[i])


@pytest.mark.parametrize("schedule", [1, 2])
def test_graph_replay_is_identical(abp, schedule):
    w = uneven(n_sets=6)
    st = torch.cuda.Stream()
    outs = []
    with abp.Ensemble(w, stream=st, schedule=schedule, steps_per_launch=20_000) as ens:
        with torch.cuda.stream(st):
            ens.set_params()
            for rep in range(3):  # direct launch, captured launch, replayed graph
                l0 = ens.launches()
                ens.reset(w.seed)
                ens.integrate(-1)
                assert ens.launches() - l0 == 2  # init + one integrator launch (direct or replayed)
                outs.append({k: v.clone() for k, v in ens.state().items()})
        st.synchronize()
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]) and torch.equal(outs[0][k], outs[2][k]), k


@pytest.mark.parametrize("n_traj", [4096, 12800, 25600])
def test_graph_replay_of_narrow_launches_is_identical(abp, n_traj):
    # narrow lockstep plans 32, 64 and 128 threads wide (warp-specialised, warp-specialised as
    # split 32-thread blocks after an occupancy check, plain): direct launch, captured launch and
    # replayed graph give the same bits
    w = W.single_set(n_traj=n_traj, n_steps=600, hist_x_bins=64)
    st = torch.cuda.Stream()
    outs = []
    with abp.Ensemble(w, stream=st, schedule=1, particles_per_thread=1, steps_per_launch=1000) as ens:
        with torch.cuda.stream(st):
            ens.set_params()
            assert ens.tiles()["narrow"] == {4096: 32, 12800: 64, 25600: 128}[n_traj]
            for rep in range(3):
                ens.reset(w.seed)
                ens.integrate(-1)
                outs.append({k: v.clone() for k, v in ens.state().items()})
        st.synchronize()
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]) and torch.equal(outs[0][k], outs[2][k]), k


def test_autotuner_choices(abp):
    w = W.sweep_grid(n_D=8, n_q=4, traj_per_set=1024, n_steps=20_000)
    with abp.Ensemble(w) as ens:
        ens.set_params()
        t = ens.tuning()
    assert t["schedule"] in (1, 2) and t["particles_per_thread"] in (1, 2, 4)
    with abp.Ensemble(w, schedule=2) as ens:
        ens.set_params()
        t = ens.tuning()
    # steps per work item from 10^3, 10^4, 10^5, capped at the longest set (2 x 10^4 here)
    assert t["schedule"] == 2 and t["steps_per_item"] in (1000, 10_000, 20_000)


def test_autotuner_weighs_the_batch(abp):
    # the load sweep (64 sets x 4,096 trajectories) fills 1.1 waves of lockstep blocks, so
    # half the second wave idles in every window; the work queue keeps every block busy and
    # is predicted (and measured, 9.82e11 against 8.26e11 particle-steps/s) faster.  On the
    # D x q sweep, nine lockstep waves deep, the two schedules run within 2% of each other at
    # two trajectories per thread (lockstep 1.02e12-1.04e12, work queue 1.0e12), and both beat
    # one and four trajectories per thread by 5% or more: the choice there is PPT 2, either
    # schedule.
    w = W.force_sweep()
    with abp.Ensemble(w) as ens:
        ens.set_params()
        assert ens.tuning()["schedule"] == 2
    big = W.sweep_grid(n_steps=20_000)  # 2,048 x 1,024 trajectories
    with abp.Ensemble(big) as ens:
        ens.set_params()
        t = ens.tuning()
        assert t["particles_per_thread"] == 2 and t["schedule"] in (1, 2)


def test_bounded_wait_reports_timeout_and_context_recovers(abp):
    w = uneven(n_sets=4)
    ref, ref_state, _ = run(abp, w, schedule=2, steps_per_launch=1000)
    with abp.Ensemble(w, schedule=2, steps_per_launch=1000) as ens:
        ens.set_params()
        abp.abp_set_wait_limit(ens.ctx, 200_000_000)  # 0.2 s
        abp.abp_test_hold_tile(ens.ctx, 0)            # tile 0 never publishes its rounds
        t0 = time.time()
        ens.integrate(-1)
        with pytest.raises(abp.AbpError) as ei:
            ens.synchronize()
        assert ei.value.status == abp.ABP_ETIMEOUT
        assert time.time() - t0 < 30
        # the context stays usable: clear the hook, start over, same result as a clean run
        abp.abp_test_hold_tile(ens.ctx, -1)
        abp.abp_set_wait_limit(ens.ctx, 0)
        ens.reset(w.seed)
        ens.integrate(-1)
        ens.synchronize()
        st = ens.state()
        for k in st:
            assert torch.equal(st[k], ref_state[k]), k


def _timed(abp, w, **kw):
    stream = torch.cuda.Stream()
    with abp.Ensemble(w, stream=stream, **kw) as ens, torch.cuda.stream(stream):
        ens.set_params()
        ens.integrate(-1)
        ens.results()
        ens.reset(w.seed)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.integrate(-1)
        ens.results()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), ens.tuning(), ens.tuning_report()


def test_autotuner_report_records_the_probe(abp):
    # with both schedules allowed, the best candidate of each -- and any within 3% of it by
    # the model -- is timed on the batch's first steps; the choice is the smallest prediction
    # among the probed candidates
    # (a step count of this process's own: choices are also kept in the tuning file beside the
    # library, and a batch met before is not probed again)
    n = 20_000 + os.getpid() % 997
    w = W.force_sweep(n_steps=n)
    with abp.Ensemble(w) as ens:
        ens.set_params()
        rep = ens.tuning_report()
        t = ens.tuning()
    probed = [c for c in rep["candidates"] if c["probe_ms"] > 0]
    assert rep["probe_steps"] > 0 and sorted(set(c["schedule"] for c in probed)) == [1, 2]
    for sch in (1, 2):
        best_model = min(c["model_ms"] for c in rep["candidates"] if c["schedule"] == sch)
        band = [c for c in rep["candidates"] if c["schedule"] == sch and c["model_ms"] <= best_model * 1.0295]
        assert all(c["probe_ms"] > 0 for c in band), (sch, band)
        assert all(c["model_ms"] <= best_model * 1.0305 for c in probed if c["schedule"] == sch)
    best = min(probed, key=lambda c: c["predicted_ms"])
    assert rep["chosen"] == {"schedule": best["schedule"], "ppt": best["ppt"], "steps": best["steps"]}
    assert (t["schedule"], t["particles_per_thread"], t["steps_per_item"]) == (best["schedule"], best["ppt"],
                                                                               best["steps"])
    assert all(c["steps"] in (1000, 10_000, n) for c in rep["candidates"])


@pytest.mark.parametrize("name", ["uneven", "single"])
def test_autotuned_choice_is_not_beaten_by_the_other_schedule(abp, name):
    # the uneven batch (512 sets, 256 to 65,536 trajectories, 10^4 to 10^6 steps) is what the
    # persistent work queue exists for; the single 4,096-trajectory set runs narrow lockstep
    # blocks.  Measured before the probe: the uneven batch got lockstep at 2.4% below the
    # work queue, the single set the work queue at a third of lockstep's rate.  The autotuned
    # run must be within 2% of the other schedule's best (at its own autotuned settings).
    w = W.uneven_batch() if name == "uneven" else W.single_set()
    t_auto, tun, rep = _timed(abp, w)
    other = 2 if tun["schedule"] == 1 else 1
    t_other, _, _ = _timed(abp, w, schedule=other)
    assert t_auto <= 1.02 * t_other, (name, t_auto, t_other, tun, rep)
