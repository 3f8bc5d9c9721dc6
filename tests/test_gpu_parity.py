"""GPU path (libabp.so through the C ABI) against the FP64 oracle.

Bars (written in each test):
  * Philox words: bit-exact.
  * Per trajectory, first 10^3 steps: |gpu - oracle| <= 1e-4 * max(|oracle|, s) with
    s = L for x, sqrt(D/gamma0) for v, q/c for e (FP32 state); 1e-9 for the FP64 state.
  * Ensemble means: within 3 standard errors; histograms: two-sample chi^2 with p > 0.01.
  * Splitting a run into several launches: bitwise identical.
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


def oracle_set(w, i, n_steps=None, **kw):
    base = w.traj_base()[i]
    return O.run_set(w.sets[i], seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i] if n_steps is None
                     else n_steps, traj_base=base, v0_mode=w.v0_mode, snapshot_every=w.snapshot_every,
                     hist_x_bins=w.hist_x_bins, hist_v_bins=w.hist_v_bins, v_lo=w.v_lo, v_hi=w.v_hi, **kw)


def ragged_batch(steps=1000, seed=21, v0_mode=1, **kw):
    sets = [W._with(D=0.1), W._with(D=0.5, q=3.0, asym=0.0), W._with(D=0.02, q=0.3, gamma0=2.0, F0=0.2),
            W._with(D=0.3, L=2.0, h=0.5, asym=0.4, c=0.5, d=2.0)]
    return W.Workload(name="ragged", sets=sets, n_traj=[300, 1, 1025, 513], n_steps=[steps, steps - 3, 10, steps],
                      dt=1e-3, seed=seed, v0_mode=v0_mode, **kw)


# --------------------------------------------------------------------------- noise

def test_philox_words_bit_exact(abp):
    rng = np.random.default_rng(7)
    n = 4096
    traj = rng.integers(0, 2**40, n, dtype=np.uint64)
    m = rng.integers(0, 2**36, n, dtype=np.uint64)
    traj[:4] = [0, 1, 2**32, 2**40 - 1]
    m[:4] = [0, 2**63, 2**32 - 1, 12345]
    seeds = [0, 1, 0xDEADBEEFCAFEF00D]
    for seed in seeds:
        t_d = torch.from_numpy(traj.view(np.int64)).cuda()
        m_d = torch.from_numpy(m.view(np.int64)).cuda()
        out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        abp.abp_philox(seed, t_d, m_d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        ref = np.array([O.noise_words(seed, int(traj[i]), int(m[i])) for i in range(n)], dtype=np.uint32)
        np.testing.assert_array_equal(got, ref)


def test_normals_match_oracle(abp):
    for seed, traj, n0 in [(0, 0, 0), (3, 12345, 1001), (2**40 + 5, 2**33 + 1, 4 * 2**30)]:
        out = torch.empty(20_003, dtype=torch.float32, device="cuda")
        abp.abp_normals(seed, traj, n0, out)
        torch.cuda.synchronize()
        z = out.cpu().numpy().astype(np.float64)
        zr = np.array([O.normal(seed, traj, n0 + i) for i in range(z.size)])
        # FP32 Box-Muller with hardware log2 / sqrt / sin / cos approximations
        np.testing.assert_allclose(z, zr, rtol=2e-5, atol=2e-5)
    out = torch.empty(1 << 22, dtype=torch.float32, device="cuda")
    abp.abp_normals(9, 77, 0, out)
    z = out.double()
    assert abs(z.mean().item()) < 4 / math.sqrt(z.numel())
    assert abs(z.var().item() - 1) < 4 * math.sqrt(2 / z.numel())


# --------------------------------------------------------------------------- per trajectory

def _compare_states(w, gpu_state, rtol, n_steps_override=None):
    base = w.traj_base()
    for i, p in enumerate(w.sets):
        if w.n_traj[i] == 0:
            continue
        n = w.n_steps[i] if n_steps_override is None else min(n_steps_override, w.n_steps[i])
        r = oracle_set(w, i, n_steps=n, want_states=True)
        sl = slice(base[i], base[i] + w.n_traj[i])
        sx, sv, se = p["L"], math.sqrt(p["D"] / p["gamma0"]) if p["D"] > 0 else 1.0, p["q"] / p["c"]
        for key, s in (("x", sx), ("v", sv), ("e", se), ("x0", sx)):
            got = gpu_state[key][sl]
            ref = r[key]
            bound = rtol * np.maximum(np.abs(ref), s)
            err = np.abs(got - ref)
            assert np.all(err <= bound), (i, key, float(np.max(err / bound)))
        # the time average follows the same trajectory
        bound = rtol * max(sv, float(np.max(np.abs(r["vbar"]))))
        assert np.all(np.abs(gpu_state["vbar"][sl] - r["vbar"]) <= bound), i


@pytest.mark.parametrize("ppt", [1, 2, 4])
def test_trajectories_first_1000_steps_fp32(abp, ppt):
    w = ragged_batch()
    with abp.Ensemble(w, particles_per_thread=ppt) as ens:
        ens.run()
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    _compare_states(w, st, rtol=1e-4)


def test_trajectories_fp64_state(abp):
    w = ragged_batch(steps=1000)
    with abp.Ensemble(w, state_fp64=True) as ens:
        ens.run()
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    _compare_states(w, st, rtol=1e-9)


def test_split_launches_are_bitwise_identical(abp):
    w = ragged_batch(steps=700, hist_x_bins=16, hist_v_bins=8, snapshot_every=97)
    with abp.Ensemble(w, steps_per_launch=10_000) as a:
        a.run()
        ra = a.results()
        sa = a.state()
    with abp.Ensemble(w, steps_per_launch=53) as b:
        b.set_params()
        for chunk in (1, 2, 5, 64, 100, 3):
            b.integrate(chunk)
        b.integrate(-1)
        rb = b.results()
        sb = b.state()
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


# --------------------------------------------------------------------------- ensemble

def _chi2_two_sample(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    keep = (a + b) > 0
    a, b = a[keep], b[keep]
    if a.size < 2:
        return 1.0
    Ka = math.sqrt(b.sum() / a.sum())
    Kb = math.sqrt(a.sum() / b.sum())
    chi2 = np.sum((Ka * a - Kb * b) ** 2 / (a + b))
    return float(stats.chi2.sf(chi2, a.size - 1))


def test_single_set_config_means_and_histogram(abp):
    # one parameter set, 4,096 trajectories x 10^4 steps, 256-bin histogram of x mod L
    w = W.single_set()
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    mom = res["moments"].numpy()[0]
    r = oracle_set(w, 0, want_states=True)
    assert abs(mom[0] - r["mean_v"]) <= 3 * r["se_v"]
    dx2 = (r["x"] - r["x0"]) ** 2
    assert abs(mom[2] - r["msd"]) <= 3 * dx2.std() / math.sqrt(dx2.size)
    assert mom[1] == pytest.approx(r["se_v"], rel=0.05)
    h_gpu = res["hist_x"].numpy()[0, 0]
    assert h_gpu.sum() == 4096
    assert _chi2_two_sample(h_gpu, r["hist_x"][0]) > 0.01
    # moments are consistent with the per-trajectory state readback
    assert mom[4] == pytest.approx(st["vbar"].sum(), rel=1e-12, abs=1e-12)
    assert mom[6] == pytest.approx((st["x"] - st["x0"]).sum(), rel=1e-9, abs=1e-9)


def test_ragged_batch_means_histograms_snapshots(abp):
    w = ragged_batch(steps=3000, hist_x_bins=32, hist_v_bins=24, snapshot_every=1000, v0_mode=1)
    w.v_lo, w.v_hi = -2.0, 2.0
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
    mom = res["moments"].numpy()
    hx = res["hist_x"].numpy()
    hv = res["hist_v"].numpy()
    assert hx.shape == (3, 4, 32) and hv.shape == (3, 4, 26)
    for i in range(w.n_sets):
        r = oracle_set(w, i)
        if w.n_traj[i] > 1:
            assert abs(mom[i, 0] - r["mean_v"]) <= 3 * r["se_v"], i
        else:  # a single trajectory has no standard error
            assert np.isfinite(mom[i, 0]) and mom[i, 1] == 0.0
        ns = O.n_snapshots(w.n_steps[i], w.snapshot_every)
        for k in range(3):
            if k < ns:
                assert hx[k, i].sum() == w.n_traj[i]
                assert hv[k, i].sum() == w.n_traj[i]
                if w.n_traj[i] >= 20:
                    assert _chi2_two_sample(hx[k, i], r["hist_x"][k]) > 0.01
                    assert _chi2_two_sample(hv[k, i], r["hist_v"][k]) > 0.01
            else:
                assert hx[k, i].sum() == 0


def test_sweep_config_sampled_sets(abp):
    # the D x q sweep shape at reduced size (all 2,048 sets, 64 trajectories, 2,000 steps):
    # sampled sets against the oracle, every set's histogram complete
    w = W.sweep_grid(traj_per_set=64, n_steps=2000)
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
    mom = res["moments"].numpy()
    assert np.all(np.isfinite(mom))
    assert np.all(res["hist_x"].numpy()[0].sum(1) == 64)
    for i in (0, 31, 700, 1024, 2047):
        r = oracle_set(w, i)
        assert abs(mom[i, 0] - r["mean_v"]) <= 3 * r["se_v"] + 1e-9, i
        assert mom[i, 2] == pytest.approx(r["msd"], rel=0.2, abs=1e-6), i


# --------------------------------------------------------------------------- edge cases

def test_edge_cases(abp):
    sets = [W._with(), W._with(D=0.0), W._with(D=0.2)]
    w = W.Workload(name="edge", sets=sets, n_traj=[0, 5, 7], n_steps=[100, 100, 0], dt=1e-3, seed=3,
                   hist_x_bins=8)
    with abp.Ensemble(w) as ens:
        ens.run()
        res = ens.results(host=True)
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    mom = res["moments"].numpy()
    assert np.all(mom[0] == 0)
    hx = res["hist_x"].numpy()[0]
    assert hx[0].sum() == 0 and hx[1].sum() == 5 and hx[2].sum() == 7
    # zero steps: state is the initial condition, time average 0
    assert np.all(st["x"][5:] == st["x0"][5:]) and np.all(st["vbar"][5:] == 0)
    # D = 0 from v0 = 0: the motion is deterministic -- compare with the oracle tightly
    r = oracle_set(w, 1, want_states=True)
    np.testing.assert_allclose(st["x"][:5], r["x"], rtol=1e-5, atol=1e-6)

    empty = W.Workload(name="empty", sets=[], n_traj=[], n_steps=[], dt=1e-3)
    with abp.Ensemble(empty) as ens:
        ens.run()
        assert ens.results(host=True)["moments"].shape == (0, 8)


def test_errors_are_reported(abp):
    w = W.single_set(n_traj=10, n_steps=10)
    with abp.Ensemble(w) as ens:
        with pytest.raises(abp.AbpError) as ei:
            ens.results()
        assert ei.value.status == abp.ABP_ESTATE
        bad = W.Workload(name="bad", sets=[W._with(L=-1.0)], n_traj=[4], n_steps=[4])
        with pytest.raises(abp.AbpError) as ei:
            abp.abp_set_params(ens.ctx, bad.sets, bad.n_traj, bad.n_steps)
        assert ei.value.status == abp.ABP_EINVAL and "L" in str(ei.value)
        with pytest.raises(abp.AbpError):
            abp.abp_set_params(ens.ctx, w.sets, [4], [2**34])
        with pytest.raises(abp.AbpError):
            abp.abp_backward(ens.ctx, None, torch.empty(6, dtype=torch.float64, device="cuda"))
    cfg = abp.make_config(w)
    cfg.dt = 0.0
    with pytest.raises(abp.AbpError):
        abp.abp_create(cfg)


def test_parameter_matrix_and_dicts_give_the_same_batch(abp):
    # abp_set_params takes the sets as dicts or as a host [sets, 9] float64 matrix (passed
    # without a copy): the same batch, the same bits
    w = ragged_batch(steps=300)
    out = []
    for form in ("dicts", "matrix"):
        with abp.Ensemble(w) as ens:
            if form == "dicts":
                abp.abp_set_params(ens.ctx, w.sets, w.n_traj, w.n_steps)
            else:
                abp.abp_set_params(ens.ctx, w.param_matrix(), np.asarray(w.n_traj), np.asarray(w.n_steps))
            ens.integrate(-1)
            st = ens.state()
            ens.synchronize()
            out.append({k: v.cpu().numpy() for k, v in st.items()})
    for k in out[0]:
        np.testing.assert_array_equal(out[0][k], out[1][k], err_msg=k)
    with abp.Ensemble(w) as ens:
        with pytest.raises(ValueError):
            abp.abp_set_params(ens.ctx, w.param_matrix()[:, :8], w.n_traj, w.n_steps)
        with pytest.raises(ValueError):
            abp.abp_set_params(ens.ctx, w.param_matrix(), w.n_traj[:-1], w.n_steps)


@pytest.mark.parametrize("scheme,noise", [(0, 0), (1, 0), (0, 1)])
def test_paired_steps_match_scalar_steps_bitwise(abp, scheme, noise):
    # One trajectory per thread runs the scalar FP32 step; two and four step trajectory pairs
    # with paired FP32 instructions, which round each half as the scalar operation.  Ragged
    # sets (odd counts leave a half of the last pair idle), step counts that are not multiples
    # of 4 (single-step heads and tails), 64-step folds, snapshots and split launches: every
    # trajectory and every histogram count must be the same bits as the scalar run.  The
    # ragged sets are followed by 150 sets of 257 trajectories, so that every lockstep launch
    # has more tiles than SMs and runs wide (a narrow launch steps one trajectory per thread
    # whatever the setting, which would compare the scalar kernel with itself).
    w = ragged_batch(steps=777, seed=23, hist_x_bins=16, hist_v_bins=8, v_lo=-2.0, v_hi=2.0, snapshot_every=97,
                     scheme=scheme, noise=noise)
    w.sets = w.sets + [W._with(D=0.05 + 0.002 * k, q=0.5 + 0.02 * k) for k in range(150)]
    w.n_traj = w.n_traj + [257] * 150
    w.n_steps = w.n_steps + [777 - (k % 5) for k in range(150)]

    def run(**kw):
        with abp.Ensemble(w, **kw) as ens:
            ens.run()
            res, st = ens.results(), ens.state()
            torch.cuda.synchronize()
            if kw.get("schedule") == 1:
                assert ens.tiles()["narrow"] == 0 and ens.tiles()["tiles"] >= 152, (kw, ens.tiles())
            return res, st

    ref_r, ref_s = run(particles_per_thread=1, schedule=1)
    for kw in (dict(particles_per_thread=2, schedule=1), dict(particles_per_thread=4, schedule=1),
               dict(particles_per_thread=2, schedule=2), dict(particles_per_thread=4, schedule=2),
               dict(particles_per_thread=2, schedule=1, steps_per_launch=53)):
        r, s = run(**kw)
        for k in ref_s:
            assert torch.equal(ref_s[k], s[k]), (kw, k)
        for k in ref_r:
            if k != "moments":  # the FP64 summation tree follows the tiles, and so PPT
                assert torch.equal(ref_r[k], r[k]), (kw, k)


def test_trajectory_ids_across_the_32_bit_boundary(abp):
    # the Philox counter carries the global trajectory id as (lo, hi) 32-bit words: a shard
    # whose ids run from 2^32 - 300 across 2^32, and one just below 2^40, must step every
    # trajectory as the oracle does (first 10^3 steps, the 1e-4 bar)
    sets = [W._with(D=0.1), W._with(D=0.3, q=2.0, asym=0.1)]
    for first in (2**32 - 300, 2**40 - 700):
        w = W.Workload(name="ids", sets=sets, n_traj=[400, 300], n_steps=[1000, 999], dt=1e-3, seed=19, v0_mode=1)
        with abp.Ensemble(w, traj_base=first) as ens:
            ens.run()
            st = {k: v.cpu().numpy() for k, v in ens.state().items()}
        base = w.traj_base()
        for i, p in enumerate(w.sets):
            r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i],
                          traj_base=first + base[i], v0_mode=w.v0_mode, want_states=True)
            sl = slice(base[i], base[i] + w.n_traj[i])
            sv = math.sqrt(p["D"] / p["gamma0"])
            for key, s in (("x", p["L"]), ("v", sv), ("e", p["q"] / p["c"]), ("x0", p["L"])):
                bound = 1e-4 * np.maximum(np.abs(r[key]), s)
                assert np.all(np.abs(st[key][sl] - r[key]) <= bound), (first, i, key)


@pytest.mark.parametrize("n_sets", [4, 4096])
def test_moments_are_the_same_bits_in_every_kind_of_output(abp, n_sets):
    # abp_reduce writes the moments into a device output directly, into a small page-locked
    # host output through its device mapping, and otherwise (pageable host memory, or 4,096
    # sets: 256 KB) through its own buffer and a copy; every route gives the same bits
    w = W.force_sweep(n_F=n_sets, traj_per_set=3, n_steps=200)
    with abp.Ensemble(w) as ens:
        ens.run()
        dev = torch.empty((n_sets, 8), dtype=torch.float64, device="cuda")
        pinned = torch.empty((n_sets, 8), dtype=torch.float64, pin_memory=True)
        pageable = torch.empty((n_sets, 8), dtype=torch.float64)
        for out in (dev, pinned, pageable):
            abp.abp_reduce(ens.ctx, out, None, None)
        torch.cuda.synchronize()
    ref = dev.cpu()
    assert torch.equal(ref, pinned) and torch.equal(ref, pageable)
    assert np.isfinite(ref.numpy()[:, 0]).all()
