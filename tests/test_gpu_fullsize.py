"""Full-size workloads in the configuration the benchmark uses (autotuned schedule and PPT),
checked on outputs the oracle can recompute: whole parameter sets, or the first trajectories
of a set (same global ids, so the same noise paths), over the full step count.

Bars: mean velocity within 3 combined standard errors (over these horizons the chaotic
frozen-noise dynamics has decorrelated GPU and oracle paths, so the two ensembles are
independent samples); for a trajectory subset, the GPU's mean of the same trajectories'
time averages against the oracle's, and the whole set's mean against the subset's;
histograms: two-sample chi^2, p > 0.01.
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


def chi2_p(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    Ka, Kb = math.sqrt(b.sum() / a.sum()), math.sqrt(a.sum() / b.sum())
    return float(stats.chi2.sf(np.sum((Ka * a - Kb * b) ** 2 / (a + b)), a.size - 1))


def test_sweep_full_size_whole_sets(abp):
    # 2,048 sets x 1,024 trajectories x 10^5 steps, as timed by the benchmark
    w = W.sweep_grid()
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
    mom = res["moments"].numpy()
    hx = res["hist_x"].numpy()[0]
    assert np.all(np.isfinite(mom)) and np.all(hx.sum(1) == 1024)
    base = w.traj_base()
    for i in (0, 1337, 2047):
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, hist_x_bins=w.hist_x_bins)
        # after 10^5 steps the frozen-noise dynamics has decorrelated the paths (it is chaotic):
        # the two ensembles are independent samples, so their errors combine
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * math.hypot(mom[i, 1], r["se_v"]), i
        assert mom[i, 3] == pytest.approx(r["d_eff"], rel=0.25, abs=1e-6), i
        assert chi2_p(hx[i].reshape(32, 8).sum(1), r["hist_x"][0].reshape(32, 8).sum(1)) > 0.01, i


def test_uneven_batch_full_size_sampled_trajectories(abp):
    # 512 sets, 256 .. 65,536 trajectories, 10^4 .. 10^6 steps (1.2e12 particle-steps)
    w = W.uneven_batch()
    with abp.Ensemble(w) as ens:
        ens.run()
        mom = ens.results(host=True)["moments"].numpy()
        vbar = ens.state()["vbar"].cpu().numpy()
    base = w.traj_base()
    longest = int(np.argmax(w.n_steps))
    largest = int(np.argmax(w.n_traj))
    for i in sorted({0, 200, longest, largest}):
        m = min(256, w.n_traj[i])
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=m, n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode)
        g = vbar[base[i]:base[i] + m]
        se_g = g.std(ddof=1) / math.sqrt(m) if m > 1 else 0.0
        assert abs(g.mean() - r["mean_v"]) <= 3 * math.hypot(se_g, r["se_v"]), (i, g.mean(), r["mean_v"])
        se = math.hypot(mom[i, 1], r["se_v"])
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * se, i


def test_large_ensemble_full_trajectory_count(abp):
    # all 67,108,864 trajectories, 2 x 10^4 of the 10^6 steps (the full length is timed by
    # `bench.py --configs snapshots`), histograms every 10^4 steps
    w = W.large_snapshots(n_steps=20_000)
    sub = 16384
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
        st = {k: a[:sub].cpu().numpy() for k, a in ens.state().items()}
    hx = res["hist_x"].numpy()[:, 0]
    hv = res["hist_v"].numpy()[:, 0]
    assert hx.shape == (2, 1024) and np.all(hx.sum(1) == w.n_traj[0]) and np.all(hv.sum(1) == w.n_traj[0])
    r = O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=sub, n_steps=w.n_steps[0], v0_mode=w.v0_mode,
                  snapshot_every=w.snapshot_every, hist_x_bins=1024, hist_v_bins=1024, v_lo=-5.0, v_hi=5.0)
    vbar = st["vbar"]
    assert abs(vbar.mean() - r["mean_v"]) <= 3 * math.hypot(vbar.std(ddof=1) / math.sqrt(sub), r["se_v"])
    se = r["se_v"] * math.sqrt(1 + sub / w.n_traj[0])
    assert abs(res["moments"].numpy()[0, 0] - r["mean_v"]) <= 3 * se
    # the final histograms of the same 16,384 trajectories (GPU state binned as the kernels bin)
    L = w.sets[0]["L"]
    xm = st["x"] - L * np.floor(st["x"] / L)
    gx = np.bincount(np.minimum((xm / L * 1024).astype(np.int64), 1023), minlength=1024)
    gv = np.bincount(np.clip(np.floor((st["v"] + 5.0) / 10.0 * 1024).astype(np.int64), 0, 1023), minlength=1024)
    assert chi2_p(gx.reshape(64, 16).sum(1), r["hist_x"][1].reshape(64, 16).sum(1)) > 0.01
    assert chi2_p(gv.reshape(64, 16).sum(1), r["hist_v"][1, :1024].reshape(64, 16).sum(1)) > 0.01
    # the whole ensemble's histograms against an oracle sample spread over all trajectory ids
    # (64 blocks of 256 trajectories at offsets i T / 64): the first 16,384 ids alone are one
    # contiguous draw, which sampled the population's x histogram at p = 0.004
    ox = np.zeros((2, 1024))
    ov = np.zeros((2, 1026))
    for i in range(64):
        rb = O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=256, n_steps=w.n_steps[0],
                       traj_base=i * (w.n_traj[0] // 64), v0_mode=w.v0_mode, snapshot_every=w.snapshot_every,
                       hist_x_bins=1024, hist_v_bins=1024, v_lo=-5.0, v_hi=5.0)
        ox += rb["hist_x"]
        ov += rb["hist_v"]
    for k in range(2):
        assert chi2_p(hx[k].reshape(64, 16).sum(1), ox[k].reshape(64, 16).sum(1)) > 0.01, k
        assert chi2_p(hv[k, :1024].reshape(64, 16).sum(1), ov[k, :1024].reshape(64, 16).sum(1)) > 0.01, k
