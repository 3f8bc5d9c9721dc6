"""The xorshift noise option (noise = 1, Marsaglia's generator of Fig. 1) on the GPU against
the FP64 oracle.

Bars: xorshift words bit-exact; per trajectory over the first 10^3 steps
|gpu - oracle| <= 1e-4 max(|oracle|, s) as for the counter-based noise; ensemble means
within 3 standard errors; trajectories and histograms bitwise the same under every schedule,
particles per thread, packing and launch split (the state carries the generator), and after
save / load; unsupported combinations refused.
"""
import math

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


def xs_batch(steps=1000, seed=51, **kw):
    sets = [W._with(D=0.1), W._with(D=0.5, q=3.0, asym=0.0), W._with(D=0.02, q=0.3, gamma0=2.0, F0=0.2),
            W._with(D=0.3, L=2.0, h=0.5, asym=0.4, c=0.5, d=2.0)]
    sets += [W._with(D=0.05 + 0.01 * i, F0=0.02 * i) for i in range(30)]  # small sets (packed)
    return W.Workload(name="xorshift", sets=sets, n_traj=[300, 1, 700, 513] + [3] * 30,
                      n_steps=[steps, steps - 3, 10, steps] + [steps] * 30, dt=1e-3, seed=seed, v0_mode=1, noise=1,
                      **kw)


def run(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res, st = ens.results(), ens.state()
        torch.cuda.synchronize()
        return res, st


def test_xorshift_words_bit_exact(abp):
    for seed, t in [(0, 0), (51, 12345), (2**40 + 7, 2**33 + 1)]:
        out = torch.empty(4096, dtype=torch.int32, device="cuda")
        abp.abp_xorshift(seed, t, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, np.array(O.xorshift_words(seed, t, 4096), dtype=np.uint32))


@pytest.mark.parametrize("ppt", [1, 2])
def test_xorshift_trajectories_first_1000_steps(abp, ppt):
    w = xs_batch()
    _, st = run(abp, w, particles_per_thread=ppt, schedule=1)
    gs = {k: a.cpu().numpy() for k, a in st.items()}
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        if w.n_traj[i] == 0:
            continue
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, want_states=True, noise=1)
        sl = slice(base[i], base[i] + w.n_traj[i])
        sv = math.sqrt(p["D"] / p["gamma0"])
        for key, sc in (("x", p["L"]), ("x0", p["L"]), ("v", sv), ("e", p["q"] / p["c"])):
            err = np.abs(gs[key][sl] - r[key]) / np.maximum(np.abs(r[key]), sc)
            assert np.all(err <= 1e-4), (i, key, float(err.max()))


def test_xorshift_ensemble_means(abp):
    sets = [W._with(D=0.1), W._with(D=0.3, F0=-0.2)]
    w = W.Workload(name="xs_means", sets=sets, n_traj=[2048, 2048], n_steps=[5000, 5000], dt=1e-3, seed=52,
                   v0_mode=0, noise=1)
    res, _ = run(abp, w)
    mom = res["moments"].cpu().numpy()
    for i in range(2):
        r = O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=2048, n_steps=5000, traj_base=w.traj_base()[i],
                      v0_mode=0, noise=1)
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * math.hypot(mom[i, 1], r["se_v"]), i


def test_xorshift_layouts_and_splits_bitwise(abp):
    w = xs_batch(steps=700, hist_x_bins=16, hist_v_bins=8, v_lo=-2.0, v_hi=2.0, snapshot_every=97)
    ref = {p: run(abp, w, particles_per_thread=p, schedule=1) for p in (1, 2)}
    for kw in (dict(particles_per_thread=1, schedule=2), dict(particles_per_thread=2, schedule=2),
               dict(particles_per_thread=2, schedule=1, steps_per_launch=53)):
        r, s = run(abp, w, **kw)
        for k in s:
            assert torch.equal(ref[1][1][k], s[k]), (kw, k)
        for k in r:  # moments follow the tiles, so they are compared at equal PPT
            want = ref[kw["particles_per_thread"]][0][k] if k == "moments" else ref[1][0][k]
            assert torch.equal(want, r[k]), (kw, k)


def test_xorshift_save_load_resumes_bitwise(abp):
    w = xs_batch(steps=600)
    with abp.Ensemble(w) as full:
        full.run()
        ref = full.state()
    with abp.Ensemble(w) as a:
        a.set_params()
        a.integrate(250)
        img = abp.abp_save(a.ctx)
    with abp.Ensemble(w) as b:
        b.set_params()
        abp.abp_load(b.ctx, img)
        b.integrate(-1)
        st = b.state()
        for k in ref:
            assert torch.equal(ref[k], st[k]), k


def test_xorshift_refuses_unsupported(abp):
    w = xs_batch(steps=100)
    for kw in (dict(state_fp64=True), dict(scheme=1)):
        with pytest.raises(abp.AbpError):
            abp.Ensemble(w, **kw)
    wc = xs_batch(steps=100, checkpoint_every=50)
    with pytest.raises(abp.AbpError):
        abp.Ensemble(wc)
