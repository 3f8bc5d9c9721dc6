"""Packed tiles: many small parameter sets (the paper's work items, one or a few
trajectories per parameter value) share blocks.  The packed layout must give bitwise the
state, moments and histograms of the one-set-per-tile layout (the work-queue schedule never
packs), and packed sets must match the FP64 oracle trajectory by trajectory."""
import math
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


def mixed_batch(seed=3, steps=1200):
    rng = np.random.default_rng(seed)
    sets, M, N = [], [], []
    for i in range(260):  # small sets, a few step counts, some empty
        sets.append(W._with(D=float(np.exp(rng.uniform(-5, 0))), F0=float(rng.uniform(-0.5, 0.5)),
                            asym=float(rng.uniform(0, 0.5))))
        M.append(int(rng.integers(0, 40)) if i % 17 else 0)
        N.append(steps if i < 200 else steps // 2)
    sets += [W._with(D=0.1), W._with(D=0.3, q=2.0)]  # two large sets
    M += [700, 300]
    N += [steps, steps - 7]
    return W.Workload(name="mixed", sets=sets, n_traj=M, n_steps=N, dt=1e-3, seed=seed, v0_mode=1,
                      hist_x_bins=16, hist_v_bins=8, v_lo=-2.0, v_hi=2.0, snapshot_every=400)


def run(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res, st, tiles = ens.results(), ens.state(), ens.tiles()
        torch.cuda.synchronize()
        return res, st, tiles


def test_packed_layout_is_bitwise_the_unpacked_one(abp):
    w = mixed_batch()
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=1)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert ta["packed"] > 0 and tb["packed"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


def test_packed_sets_against_oracle(abp):
    w = mixed_batch(seed=4, steps=1000)
    res, st, t = run(abp, w, schedule=1, particles_per_thread=1)
    assert t["packed"] > 0
    gs = {k: a.cpu().numpy() for k, a in st.items()}
    hx = res["hist_x"].cpu().numpy()
    base = w.traj_base()
    checked = 0
    for i in range(0, 200, 7):
        if w.n_traj[i] == 0:
            continue
        p = w.sets[i]
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                      v0_mode=w.v0_mode, want_states=True, snapshot_every=w.snapshot_every, hist_x_bins=16)
        sl = slice(base[i], base[i] + w.n_traj[i])
        sv = math.sqrt(p["D"] / p["gamma0"])
        for key, sc in (("x", p["L"]), ("x0", p["L"]), ("v", sv), ("e", p["q"] / p["c"])):
            err = np.abs(gs[key][sl] - r[key]) / np.maximum(np.abs(r[key]), sc)
            assert np.all(err <= 1e-4), (i, key, err.max())
        bound = 1e-4 * max(sv, float(np.max(np.abs(r["vbar"]))))
        assert np.all(np.abs(gs["vbar"][sl] - r["vbar"]) <= bound), i
        assert np.all(hx[:, i].sum(1) == w.n_traj[i])
        mv = res["moments"][i, 0].item()
        if w.n_traj[i] > 1:  # mean over the same paths: FP32 against FP64 only
            assert abs(mv - r["mean_v"]) <= 1e-4 * max(1.0, abs(r["mean_v"]))
        checked += 1
    assert checked >= 10


def test_packed_zero_step_sets_snapshot_initial_state(abp):
    sets = [W._with(D=0.1 * (i + 1)) for i in range(6)]
    w = W.Workload(name="zero", sets=sets, n_traj=[3, 0, 5, 1, 7, 2], n_steps=[0] * 6, dt=1e-3, seed=8, v0_mode=1,
                   hist_x_bins=8, hist_v_bins=4, v_lo=-1.0, v_hi=1.0)
    res, st, t = run(abp, w, schedule=1, particles_per_thread=1)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert t["packed"] == 1 and tb["packed"] == 0
    assert res["hist_x"].cpu().numpy()[0].sum(1).tolist() == w.n_traj
    assert res["hist_v"].cpu().numpy()[0].sum(1).tolist() == w.n_traj
    for k in st:
        assert torch.equal(st[k], sb[k]), k
    for k in res:
        assert torch.equal(res[k], rb[k]), k


@pytest.mark.parametrize("n_traj,ppt", [(4096, 1), (4096, 2), (777, 1)])
def test_narrow_launch_is_bitwise_the_wide_one(abp, n_traj, ppt):
    # a batch with fewer tiles than SMs runs narrow blocks; the work queue never does
    w = W.single_set(n_traj=n_traj, n_steps=900, hist_x_bins=32)
    w.hist_v_bins, w.v_lo, w.v_hi, w.snapshot_every = 16, -2.0, 2.0, 300
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=ppt)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=ppt)
    assert ta["narrow"] in (32, 64, 128, 256) and tb["narrow"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


def test_narrow_packed_items_against_wide(abp):
    # 300 one-trajectory work items: two packed tiles, launched narrow
    w = W.force_sweep(n_F=300, traj_per_set=1, n_steps=640)
    w.hist_x_bins = 8
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=1)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert ta["packed"] == 2 and ta["narrow"] > 0 and tb["packed"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


@pytest.mark.parametrize("n_traj,scheme", [(4096, 0), (777, 0), (4096, 1), (12800, 0), (12800, 1), (25600, 0)])
def test_warp_specialised_narrow_launch_is_bitwise_the_wide_one(abp, n_traj, scheme):
    # narrow lockstep blocks of 32 stepping threads run warp-specialised (three producer warps
    # draw the noise into a shared-memory ring of 64-step slots; 777 trajectories leave a ragged
    # last block); a plan of 64-thread blocks (12,800 trajectories) runs as twice as many
    # warp-specialised 32-thread ones, a plan of 128-thread blocks (25,600) on the plain narrow
    # kernel.  Launch windows (250 steps), snapshots (every 77 steps) and the run's end (1,003
    # steps) fall inside slots; state, histograms and moments must be the work queue's bits (it
    # never narrows).
    w = W.single_set(n_traj=n_traj, n_steps=1003, hist_x_bins=32)
    w.hist_v_bins, w.v_lo, w.v_hi, w.snapshot_every, w.scheme = 16, -2.0, 2.0, 77, scheme
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=1, steps_per_launch=250)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert ta["narrow"] == {12800: 64, 25600: 128}.get(n_traj, 32) and tb["narrow"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


def test_narrow_plan_whose_split_blocks_do_not_fit_is_bitwise_the_wide_one(abp):
    # 40 tiles planned 64 wide would become 320 warp-specialised blocks, but with 8,192 + 8,194
    # histogram bins beside the 48 KB ring at most two fit on an SM (304 at once): the launch
    # keeps the plain narrow kernel; either way the bits are the work queue's
    w = W.single_set(n_traj=40 * 256, n_steps=300, hist_x_bins=8192)
    w.hist_v_bins, w.v_lo, w.v_hi, w.snapshot_every = 8192, -2.0, 2.0, 100
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=1)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert ta["tiles"] == 40 and ta["narrow"] == 64 and tb["narrow"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


@pytest.mark.parametrize("n_items,scheme,noise", [(16384, 0, 0), (16384, 1, 0), (16384, 0, 1), (32768, 0, 0)])
def test_narrow_packed_wider_blocks_are_bitwise_the_wide_ones(abp, n_items, scheme, noise):
    # 16,384 one-trajectory work items fill 64 packed tiles, planned as 64-thread narrow blocks
    # and run as 32-thread warp-specialised ones; 32,768 fill 128, planned 128 wide (the plain
    # narrow kernel); histograms of packed sets go to global memory at every snapshot, and the
    # launch windows and snapshots fall off the counter blocks
    w = W.force_sweep(n_F=n_items, traj_per_set=1, n_steps=650)
    w.hist_x_bins, w.hist_v_bins, w.v_lo, w.v_hi, w.snapshot_every = 8, 4, -2.0, 2.0, 97
    w.scheme, w.noise = scheme, noise
    ra, sa, ta = run(abp, w, schedule=1, particles_per_thread=1, steps_per_launch=300)
    rb, sb, tb = run(abp, w, schedule=2, particles_per_thread=1)
    assert ta["packed"] == n_items // 256 and ta["narrow"] == {16384: 64, 32768: 128}[n_items] and tb["packed"] == 0
    for k in sa:
        assert torch.equal(sa[k], sb[k]), k
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k


def test_warp_specialised_wait_reports_timeout_and_context_recovers(abp):
    # the test hook keeps tile 0's producer warps from handing over any noise: its stepping
    # warps wait until the (0.2 s) limit expires, the launch ends with ABP_ETIMEOUT, and the
    # context gives a clean run's bits after a reset
    w = W.single_set(n_traj=4096, n_steps=500)
    _, ref, _ = run(abp, w, schedule=1, particles_per_thread=1)
    with abp.Ensemble(w, schedule=1, particles_per_thread=1) as ens:
        ens.set_params()
        assert ens.tiles()["narrow"] == 32
        abp.abp_set_wait_limit(ens.ctx, 200_000_000)
        abp.abp_test_hold_tile(ens.ctx, 0)
        t0 = time.time()
        ens.integrate(-1)
        with pytest.raises(abp.AbpError) as ei:
            ens.synchronize()
        assert ei.value.status == abp.ABP_ETIMEOUT
        assert time.time() - t0 < 30
        abp.abp_test_hold_tile(ens.ctx, -1)
        abp.abp_set_wait_limit(ens.ctx, 0)
        ens.reset(w.seed)
        ens.integrate(-1)
        ens.synchronize()
        st = ens.state()
        for k in st:
            assert torch.equal(st[k], ref[k]), k
