"""The remaining workload shapes against the oracle: large-ensemble snapshots (1,024-bin
histograms of x mod L and of v every 2,000 steps), the FP64-state precision reference, and
the mean-velocity-versus-load sweep of the paper's Fig. 2."""
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


def _chi2_two_sample(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    Ka, Kb = math.sqrt(b.sum() / a.sum()), math.sqrt(a.sum() / b.sum())
    chi2 = np.sum((Ka * a - Kb * b) ** 2 / (a + b))
    return float(stats.chi2.sf(chi2, a.size - 1))


def test_snapshot_histograms_large_ensemble_shape(abp):
    w = W.large_snapshots(n_traj=1 << 16, n_steps=20_000, snapshot_every=2000)
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    hx = res["hist_x"].numpy()[:, 0]
    hv = res["hist_v"].numpy()[:, 0]
    assert hx.shape == (10, 1024) and hv.shape == (10, 1026)
    assert np.all(hx.sum(1) == w.n_traj[0]) and np.all(hv.sum(1) == w.n_traj[0])
    # the oracle on the first 4,096 trajectories (same ids, same noise)
    sub = 4096
    r = O.run_set(w.sets[0], seed=w.seed, dt=w.dt, n_traj=sub, n_steps=w.n_steps[0], v0_mode=w.v0_mode,
                  snapshot_every=w.snapshot_every, hist_x_bins=1024, hist_v_bins=1024, v_lo=-5.0, v_hi=5.0,
                  want_states=True)
    for k in (0, 4, 9):  # snapshots at 2,000, 10,000 and 20,000 steps, bins merged by 16
        gx = hx[k].reshape(64, 16).sum(1)
        ox = r["hist_x"][k].reshape(64, 16).sum(1)
        assert _chi2_two_sample(gx, ox) > 0.01, k
        gv = hv[k, :1024].reshape(64, 16).sum(1)
        ov = r["hist_v"][k, :1024].reshape(64, 16).sum(1)
        assert _chi2_two_sample(gv, ov) > 0.01, k
    # the mean velocity of the whole ensemble against the oracle's subset
    se = r["se_v"] * math.sqrt(1 + sub / w.n_traj[0])
    assert abs(res["moments"].numpy()[0, 0] - r["mean_v"]) <= 3.5 * se


def test_fp32_state_against_fp64_state(abp):
    # same noise, same initial condition: two integrations of the same sample paths.  Their
    # ensemble statistics must agree within the statistical error (the bar GPU vs oracle
    # uses), and most individual trajectories must stay together.
    w = W.large_snapshots(n_traj=1 << 15, n_steps=10_000, snapshot_every=5000)
    out = {}
    for fp64 in (False, True):
        with abp.Ensemble(w, state_fp64=fp64) as ens:
            ens.run()
            st = ens.state()
            out[fp64] = (ens.results(host=True)["moments"].numpy()[0], st["x"].cpu().numpy(), st["x0"].cpu().numpy())
    m32, x32, _ = out[False]
    m64, x64, x0 = out[True]
    assert abs(m32[0] - m64[0]) <= 3 * m64[1]
    dx2 = (x64 - x0) ** 2
    assert abs(m32[2] - m64[2]) <= 3 * dx2.std() / math.sqrt(dx2.size)
    assert np.median(np.abs(x32 - x64)) < 1e-3


def test_force_sweep_against_oracle(abp):
    w = W.force_sweep(n_F=16, traj_per_set=512, n_steps=5000)
    with abp.Ensemble(w) as ens:
        ens.run()
        mom = ens.results(host=True)["moments"].numpy()
    base = w.traj_base()
    for i in (0, 5, 10, 15):
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode)
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * r["se_v"], i
    # a strong load drags the particles along: <v> has the sign of F0 at the ends of the range
    assert mom[0, 0] < 0 < mom[-1, 0]
