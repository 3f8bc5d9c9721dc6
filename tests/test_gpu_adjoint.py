"""Pathwise adjoint (abp_backward) against the oracle's FP64 tangent-linear gradient.

The oracle's tangent-linear is itself pinned to FP64 central differences with common
random numbers (tests/test_oracle_pins.py).  Bar: the GPU adjoint of the mean velocity
agrees with it within 1e-3 relative (of the largest gradient component of the set),
on runs short enough that the FP32 and FP64 trajectories stay together.
"""
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


def batch(K=500, v0_mode=1):
    sets = [W._with(D=0.05), W._with(D=0.2, q=2.0, asym=0.1, gamma0=1.5), W._with(D=0.1, F0=0.3, c=0.3, d=0.7)]
    return W.Workload(name="adj", sets=sets, n_traj=[256, 100, 300], n_steps=[2000, 1900, 777], dt=1e-3, seed=31,
                      v0_mode=v0_mode, checkpoint_every=K)


def oracle_grads(w):
    base = w.traj_base()
    out = []
    for i, p in enumerate(w.sets):
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, want_grad=True)
        out.append(r["grad"])
    return np.array(out)


@pytest.mark.parametrize("K,v0_mode", [(500, 1), (64, 0), (333, 1)])
def test_adjoint_matches_oracle_tangent_linear(abp, K, v0_mode):
    w = batch(K, v0_mode)
    with abp.Ensemble(w) as ens:
        ens.run()
        g = ens.backward(host=True).numpy()
    ref = oracle_grads(w)
    for i in range(w.n_sets):
        scale = np.max(np.abs(ref[i]))
        np.testing.assert_allclose(g[i], ref[i], rtol=1e-3, atol=1e-3 * scale, err_msg="set %d" % i)


def test_adjoint_weights_and_device_outputs(abp):
    w = batch()
    with abp.Ensemble(w) as ens:
        ens.run()
        g1 = ens.backward()
        wt = torch.tensor([2.0, -1.0, 0.5], dtype=torch.float64, device="cuda")
        g2 = ens.backward(wt)
        torch.cuda.synchronize()
    np.testing.assert_allclose(g2.cpu().numpy(), g1.cpu().numpy() * np.array([[2.0], [-1.0], [0.5]]), rtol=1e-12)


def test_adjoint_requires_checkpoints_and_completion(abp):
    w = batch(K=0)
    with abp.Ensemble(w) as ens:
        ens.run()
        with pytest.raises(abp.AbpError) as ei:
            ens.backward()
        assert ei.value.status == abp.ABP_ESTATE
    w = batch(K=100)
    with abp.Ensemble(w) as ens:
        ens.set_params()
        ens.integrate(50)
        with pytest.raises(abp.AbpError) as ei:
            ens.backward()
        assert ei.value.status == abp.ABP_ESTATE


def test_autograd_function(abp):
    w = batch()
    theta = torch.tensor([[s[k] for k in abp.GRAD_PARAMS] for s in w.sets], dtype=torch.float64, requires_grad=True)
    mv = abp.MeanVelocity.apply(theta, w)
    mv.sum().backward()
    ref = oracle_grads(w)
    np.testing.assert_allclose(theta.grad.numpy(), ref, rtol=1e-3, atol=1e-3 * np.abs(ref).max())


@pytest.mark.parametrize("window", [500, 1000])
def test_windowed_adjoint_matches_oracle(abp, window):
    # 2,000 steps: the FP32 and FP64 paths stay together, so the windowed derivatives must
    # agree as the full ones do (1e-3 of the largest component)
    sets = [W._with(D=0.05), W._with(D=0.2, q=2.0, asym=0.1)]
    w = W.Workload(name="adj_win", sets=sets, n_traj=[512, 300], n_steps=[2000, 1800], dt=1e-3, seed=33, v0_mode=1,
                   checkpoint_every=500)
    with abp.Ensemble(w) as ens:
        ens.run()
        g = ens.backward(host=True, window=window).numpy()
        full = ens.backward(host=True).numpy()
        same = ens.backward(host=True, window=2000).numpy()
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, want_grad=True, grad_window=window)
        scale = np.max(np.abs(r["grad"]))
        assert np.max(np.abs(g[i] - r["grad"])) <= 1e-3 * scale, (i, g[i], r["grad"])
    np.testing.assert_array_equal(same, full)  # a window past the run is the full adjoint
    for bad in (-1, 250, 777):
        with pytest.raises(abp.AbpError):
            with abp.Ensemble(w) as e2:
                e2.run()
                e2.backward(window=bad)


def test_windowed_adjoint_long_horizon(abp):
    # 8,000 steps (t = 8): chaos has separated some FP32 paths from their FP64 twins, so the
    # two windowed estimates are compared within their statistical error (per-trajectory
    # spread of the oracle's windowed tangents), and both stay bounded while the full pathwise
    # derivative has grown by ~e^{0.46 t}
    p = W._with(D=0.05)
    w = W.Workload(name="adj_long", sets=[p], n_traj=[2048], n_steps=[8000], dt=1e-3, seed=34, v0_mode=1,
                   checkpoint_every=500)
    with abp.Ensemble(w) as ens:
        ens.run()
        g = ens.backward(host=True, window=1500).numpy()[0]
        full = ens.backward(host=True).numpy()[0]
    r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=2048, n_steps=8000, v0_mode=1, want_traj_grad=True,
                  grad_window=1500)
    se = r["dvbar"].std(axis=0, ddof=1) / np.sqrt(2048)
    assert np.all(np.abs(g - r["grad"]) <= 3 * np.sqrt(2) * se + 1e-3 * np.max(np.abs(r["grad"]))), (g, r["grad"], se)
    assert np.max(np.abs(g)) < 0.1 * np.max(np.abs(full))


@pytest.mark.parametrize("K,v0_mode,window", [(250, 1, 0), (64, 0, 0), (250, 1, 500)])
def test_adjoint_per_trajectory_matches_oracle_tangent(abp, K, v0_mode, window):
    # every trajectory's derivative d vbar_i / d theta (no averaging, so errors of opposite
    # sign cannot cancel) against the oracle's FP64 tangent of the same trajectory, over
    # 1,000 steps where the FP32 and FP64 paths stay together: |gpu - oracle| <=
    # 1e-3 max(|oracle|, s_j), s_j = the root mean square of component j over the set
    sets = [W._with(D=0.05), W._with(D=0.2, q=2.0, asym=0.1, gamma0=1.5), W._with(D=0.1, F0=0.3, c=0.3, d=0.7)]
    w = W.Workload(name="adj_traj", sets=sets, n_traj=[1000, 513, 700], n_steps=[1000, 1000, 750], dt=1e-3, seed=35,
                   v0_mode=v0_mode, checkpoint_every=K)
    with abp.Ensemble(w) as ens:
        ens.run()
        g = ens.backward(host=True, window=window).numpy()
        dv = ens.traj_grad(host=True).numpy()
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, want_traj_grad=True, grad_window=window)
        ref = r["dvbar"]
        sl = slice(base[i], base[i] + w.n_traj[i])
        s = np.sqrt(np.mean(ref**2, axis=0))
        bound = 1e-3 * np.maximum(np.abs(ref), s)
        ratio = np.abs(dv[sl] - ref) / bound
        assert np.all(ratio <= 1.0), (i, float(ratio.max()), np.unravel_index(ratio.argmax(), ratio.shape))
        # the set gradient (unit weights) is the mean of the trajectories' derivatives
        np.testing.assert_allclose(dv[sl].mean(axis=0), g[i], rtol=1e-9, atol=1e-12 * np.abs(g[i]).max())


def test_adjoint_at_zero_noise(abp):
    # D = 0: sigma = sqrt(2 D dt) has no derivative there, so the D-component is NaN (in the
    # set gradient and for every trajectory); the other components are those of the
    # deterministic model and match the oracle's tangent
    sets = [W._with(D=0.0, F0=0.1), W._with(D=0.1)]
    w = W.Workload(name="adj_d0", sets=sets, n_traj=[300, 300], n_steps=[800, 800], dt=1e-3, seed=36, v0_mode=0,
                   checkpoint_every=200)
    with abp.Ensemble(w) as ens:
        ens.run()
        g = ens.backward(host=True).numpy()
        dv = ens.traj_grad(host=True).numpy()
    r = O.run_set(sets[0], seed=w.seed, dt=w.dt, n_traj=300, n_steps=800, v0_mode=0, want_traj_grad=True)
    assert np.isnan(g[0, 0]) and np.isnan(r["grad"][0]) and np.all(np.isnan(dv[:300, 0]))
    assert np.all(np.isfinite(g[0, 1:])) and np.all(np.isfinite(g[1]))
    np.testing.assert_allclose(g[0, 1:], r["grad"][1:], rtol=1e-3, atol=1e-3 * np.abs(r["grad"][1:]).max())
    # the readout is refused once the batch has been restarted
    with abp.Ensemble(w) as ens:
        ens.run()
        ens.backward()
        ens.reset()
        with pytest.raises(abp.AbpError) as ei:
            ens.traj_grad()
        assert ei.value.status == abp.ABP_ESTATE


@pytest.mark.parametrize("K,window,ppt", [(64, 0, 2), (256, 512, 2), (1000, 0, 2), (256, 0, 1), (256, 512, 4)])
def test_philox_handoff_gives_the_same_bits(abp, K, window, ppt, monkeypatch):
    # checkpoint intervals of whole 8-step sub-chunks let level 1 hand its Philox blocks to the
    # reverse sweep (ABP_ADJ_HANDOFF_BYTES unset: within half the free memory); 0 bytes makes
    # the reverse sweep draw them again.  Ragged sets (odd sizes: a thread with one trajectory;
    # step counts with a partial last chunk and a short last segment): every set gradient and
    # every trajectory's derivative bit for bit the same (1, 2 or 4 trajectories per thread in
    # the forward: 1, 2 or 4 adjoint blocks per tile, the hand-off laid out by block)
    sets = [W._with(D=0.05), W._with(D=0.2, q=2.0, asym=0.1, gamma0=1.5), W._with(D=0.1, F0=0.3, c=0.3, d=0.7)]
    w = W.Workload(name="handoff", sets=sets, n_traj=[1000, 257, 3], n_steps=[2051, 1900, 1024], dt=1e-3, seed=37,
                   v0_mode=1, checkpoint_every=K)
    out = {}
    for tag, env in (("handoff", None), ("redraw", "0")):
        if env is None:
            monkeypatch.delenv("ABP_ADJ_HANDOFF_BYTES", raising=False)
        else:
            monkeypatch.setenv("ABP_ADJ_HANDOFF_BYTES", env)
        with abp.Ensemble(w, schedule=1, particles_per_thread=ppt) as ens:
            ens.run()
            out[tag] = (ens.backward(host=True, window=window).numpy(), ens.traj_grad(host=True).numpy())
    np.testing.assert_array_equal(out["handoff"][0], out["redraw"][0])
    np.testing.assert_array_equal(out["handoff"][1], out["redraw"][1])
    assert np.all(np.isfinite(out["handoff"][0]))
