"""The stochastic Heun variant of the step (scheme = 1) on the GPU against the FP64 oracle.

Bars, as for the Euler-Maruyama path:
  * per trajectory, first 10^3 steps: |gpu - oracle| <= 1e-4 max(|oracle|, s), s = L for x,
    sqrt(D/gamma0) for v, q/c for e;
  * ensemble means within 3 standard errors of the oracle's, at a step 5x the default;
  * the free passive velocity's stationary variance matches the Heun map's closed form
    (and differs from Euler-Maruyama's by more than the statistical error);
  * schedules, particles per thread and split launches: bitwise identical.
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


def heun_batch(steps=1000, dt=1e-3, seed=31, **kw):
    sets = [W._with(D=0.1), W._with(D=0.5, q=3.0, asym=0.0), W._with(D=0.02, q=0.3, gamma0=2.0, F0=0.2),
            W._with(D=0.3, L=2.0, h=0.5, asym=0.4, c=0.5, d=2.0), W._with(D=0.15, F0=-0.26, asym=0.25)]
    return W.Workload(name="heun", sets=sets, n_traj=[300, 1, 700, 513, 40], n_steps=[steps, steps - 3, 10, steps, steps],
                      dt=dt, seed=seed, v0_mode=1, scheme=1, **kw)


def oracle_set(w, i, **kw):
    return O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i],
                     traj_base=w.traj_base()[i], v0_mode=w.v0_mode, scheme=1, **kw)


def run(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res, st = ens.results(), ens.state()
        torch.cuda.synchronize()
        return res, st


@pytest.mark.parametrize("ppt", [1, 2])
def test_heun_trajectories_first_1000_steps(abp, ppt):
    w = heun_batch()
    _, st = run(abp, w, particles_per_thread=ppt, schedule=1)
    gs = {k: a.cpu().numpy() for k, a in st.items()}
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        r = oracle_set(w, i, want_states=True)
        sl = slice(base[i], base[i] + w.n_traj[i])
        sv = math.sqrt(p["D"] / p["gamma0"])
        for key, sc in (("x", p["L"]), ("x0", p["L"]), ("v", sv), ("e", p["q"] / p["c"])):
            err = np.abs(gs[key][sl] - r[key]) / np.maximum(np.abs(r[key]), sc)
            assert np.all(err <= 1e-4), (i, key, float(err.max()))
        bound = 1e-4 * max(sv, float(np.max(np.abs(r["vbar"]))))
        assert np.all(np.abs(gs["vbar"][sl] - r["vbar"]) <= bound), i


def test_heun_ensemble_means_at_large_step(abp):
    # dt = 5e-3, 4,000 steps (t = 20): mean velocity and D_eff within 3 SE of the oracle's
    sets = [W._with(D=0.1), W._with(D=0.3, F0=-0.2), W._with(D=0.05, asym=0.0)]
    w = W.Workload(name="heun_means", sets=sets, n_traj=[2048] * 3, n_steps=[4000] * 3, dt=5e-3, seed=32,
                   v0_mode=0, scheme=1, hist_x_bins=32)
    res, _ = run(abp, w)
    mom = res["moments"].cpu().numpy()
    hx = res["hist_x"].cpu().numpy()[0]
    for i in range(3):
        r = oracle_set(w, i, hist_x_bins=32)
        se = math.hypot(mom[i, 1], r["se_v"])
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * se, (i, mom[i, 0], r["mean_v"], se)
        assert hx[i].sum() == 2048
        # histograms of x mod L: two-sample chi^2, p > 0.01
        a, b = hx[i].astype(float), r["hist_x"][0].astype(float)
        keep = (a + b) > 0
        chi2 = float(np.sum((a[keep] - b[keep]) ** 2 / (a[keep] + b[keep])))
        assert stats.chi2.sf(chi2, int(keep.sum()) - 1) > 0.01, chi2


def test_heun_free_velocity_variance_closed_form(abp):
    # d = 0, h = 0, F0 = 0: v' = a v + b z, a = 1 - g dt + (g dt)^2/2, b = sqrt(2 D dt)(1 - g dt/2);
    # from v0 = 0 after N steps Var v = b^2 (1 - a^{2N}) / (1 - a^2)
    D, g, dt, N, M = 0.3, 2.0, 0.1, 400, 1 << 18
    w = W.Workload(name="heun_ou", sets=[W._with(d=0.0, h=0.0, F0=0.0, D=D, gamma0=g)], n_traj=[M], n_steps=[N],
                   dt=dt, seed=33, v0_mode=0, scheme=1)
    _, st = run(abp, w)
    v = st["v"].cpu().numpy()
    a = 1 - g * dt + 0.5 * (g * dt) ** 2
    b2 = 2 * D * dt * (1 - 0.5 * g * dt) ** 2
    var_heun = b2 * (1 - a ** (2 * N)) / (1 - a**2)
    rho = 1 - g * dt
    var_em = 2 * D * dt * (1 - rho ** (2 * N)) / (1 - rho**2)
    tol = 4 * var_heun * math.sqrt(2.0 / M)
    assert abs(np.mean(v**2) - var_heun) < tol
    assert abs(var_em - var_heun) > 3 * tol


def test_heun_schedules_ppt_and_split_launches_bitwise(abp):
    # trajectories and histogram counts: the same bits under every schedule, PPT and launch
    # split; moments too at equal PPT (the tiles, and so the FP64 summation tree, follow PPT)
    w = heun_batch(steps=700, hist_x_bins=16, hist_v_bins=8, v_lo=-2.0, v_hi=2.0, snapshot_every=97)
    ref = {p: run(abp, w, particles_per_thread=p, schedule=1) for p in (1, 2)}
    for kw in (dict(particles_per_thread=2, schedule=1), dict(particles_per_thread=1, schedule=2),
               dict(particles_per_thread=2, schedule=2), dict(particles_per_thread=2, schedule=1, steps_per_launch=53)):
        r, s = run(abp, w, **kw)
        ref_r, ref_s = ref[kw["particles_per_thread"]]
        for k in s:
            assert torch.equal(ref[1][1][k], s[k]), (kw, k)
        for k in r:
            assert torch.equal(ref_r[k], r[k]), (kw, k)
            if k != "moments":
                assert torch.equal(ref[1][0][k], r[k]), (kw, k)


def test_heun_differs_from_euler_maruyama_and_rejects_unsupported(abp):
    w = heun_batch(steps=200)
    _, sh = run(abp, w)
    we = heun_batch(steps=200)
    we.scheme = 0
    _, se = run(abp, we)
    assert not torch.equal(sh["v"], se["v"])
    assert torch.equal(sh["x0"], se["x0"])  # same initial condition
    for bad in (dict(state_fp64=True),):
        with pytest.raises(abp.AbpError):
            abp.Ensemble(w, **bad)
    wc = heun_batch(steps=200, checkpoint_every=100)
    with pytest.raises(abp.AbpError):
        abp.Ensemble(wc)
