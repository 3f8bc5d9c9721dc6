"""The integrator instantiations the benchmark runs -- wide lockstep launches (one block of 256
threads per tile, two or four trajectories per thread on paired FP32 instructions) and the
persistent work queue -- against the FP64 oracle trajectory by trajectory, and against each
other bit for bit.

A lockstep batch with fewer tiles than SMs is launched narrow (one trajectory per thread), so
the batch here has 160 parameter sets of 512 trajectories: 160 tiles at two and at four
trajectories per thread, 320 at one, more than the 152 SMs of a GB300 in every case, and each
launch asserts that it ran wide.  Sets mix D, q and the asymmetry a; their step counts
(992..1000) are mostly not multiples of the four steps of a Philox block, and histograms are
taken every 250 steps.

Bars (written in the tests):
  * every trajectory, after its 992..1000 steps (the first 10^3 steps of Sec. 2's model,
    Eqs. (ereservoir), (velocity), (pot), stepped as in Fig. 1): |gpu - oracle| <=
    1e-4 max(|oracle|, s) + 3 |oracle' - oracle|, s = L for x, the larger of the thermal
    speed sqrt(D / gamma0) and the depot-driven speed v* = sqrt(q / gamma0 - c / d) for v,
    q / c for e.  oracle' is the oracle run with every noise increment (and the random
    initial velocity) larger by a relative 1e-6 -- D raised by 2e-6 D --, the accuracy of the
    FP32 Box-Muller transform: the term is the change that an error of that size makes to
    the exact trajectory, so it only matters for the few trajectories whose dynamics
    amplifies such errors past the 1e-4 bar (passing close to a barrier top of an
    asymmetric potential), and at least 99.9% of the trajectories must also meet the plain
    1e-4 bar without it;
  * lockstep at 1, 2 and 4 trajectories per thread and the work queue at 1, 2 and 4: the
    same bits for every trajectory and every histogram count; moments bitwise between the
    two schedules at equal trajectories per thread (equal tiles).
Run for the counter-based Euler-Maruyama step, the stochastic Heun step and xorshift noise.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1104_2499_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_SETS, M = 160, 512


@pytest.fixture(scope="module")
def abp():
    from paper_1104_2499_gb300 import abp as A
    from paper_1104_2499_gb300 import build as B

    B.build()
    A.lib()
    return A


def wide_batch(scheme=0, noise=0):
    rng = np.random.default_rng(1601)
    D = np.exp(rng.uniform(math.log(0.01), math.log(0.5), N_SETS))
    q = np.exp(rng.uniform(math.log(0.3), math.log(5.0), N_SETS))
    a = rng.uniform(0.0, 0.5, N_SETS)
    steps = rng.integers(992, 1001, N_SETS)
    sets = [W.params(D=float(D[i]), q=float(q[i]), asym=float(a[i])) for i in range(N_SETS)]
    return W.Workload(name="wide", sets=sets, n_traj=[M] * N_SETS, n_steps=[int(n) for n in steps], dt=1e-3,
                      seed=77, v0_mode=1, hist_x_bins=32, hist_v_bins=16, v_lo=-4.0, v_hi=4.0, snapshot_every=250,
                      scheme=scheme, noise=noise)


def run(A, w, **kw):
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        res = ens.results()
        st = ens.state()
        torch.cuda.synchronize()
        return res, st, ens.tiles(), ens.tuning()


MODES = {"em": (0, 0), "heun": (1, 0), "xorshift": (0, 1)}


# Relative size of the noise perturbation that measures a trajectory's conditioning: the
# accuracy of the FP32 Box-Muller transform (hardware log2, sin/cos and square root).
NOISE_EPS = 1e-6


@pytest.fixture(scope="module")
def oracle_states():
    cache = {}

    def get(mode):
        if mode not in cache:
            w = wide_batch(*MODES[mode])
            base = w.traj_base()
            out = []
            for i, p in enumerate(w.sets):
                kw = dict(seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i], traj_base=base[i],
                          v0_mode=w.v0_mode, scheme=w.scheme, noise=w.noise, want_states=True)
                ref = O.run_set(p, **kw)
                pert = O.run_set(dict(p, D=p["D"] * (1.0 + 2.0 * NOISE_EPS)), **kw)
                out.append((ref, pert))
            cache[mode] = out
        return cache[mode]

    return get


def velocity_scale(p):
    """The model's velocity scale: the thermal speed sqrt(D / gamma0), or the speed
    v* = sqrt(q / gamma0 - c / d) at which the depot's pumping balances friction (Sec. 2),
    whichever is larger."""
    return max(math.sqrt(p["D"] / p["gamma0"]), math.sqrt(max(p["q"] / p["gamma0"] - p["c"] / p["d"], 0.0)))


def assert_trajectories_match_oracle(w, st, ref, rtol=1e-4):
    base = w.traj_base()
    plain_ok = total = 0
    for i, p in enumerate(w.sets):
        r, rp = ref[i]
        sl = slice(base[i], base[i] + w.n_traj[i])
        scale = {"x": p["L"], "x0": p["L"], "v": velocity_scale(p), "e": p["q"] / p["c"]}
        ok = np.ones(w.n_traj[i], dtype=bool)
        for key, s in scale.items():
            err = np.abs(st[key][sl] - r[key])
            bar = rtol * np.maximum(np.abs(r[key]), s)
            cond = 3.0 * np.abs(rp[key] - r[key])
            ratio = err / (bar + cond)
            assert np.all(ratio <= 1.0), (i, key, float(ratio.max()), int(ratio.argmax()))
            ok &= err <= bar
        bound = rtol * max(scale["v"], float(np.max(np.abs(r["vbar"])))) + 3.0 * np.abs(rp["vbar"] - r["vbar"])
        assert np.all(np.abs(st["vbar"][sl] - r["vbar"]) <= bound), i
        plain_ok += int(ok.sum())
        total += w.n_traj[i]
    assert plain_ok >= 0.999 * total, (plain_ok, total)
    return plain_ok / total


@pytest.mark.parametrize("mode", list(MODES))
def test_wide_launches_match_oracle_per_trajectory_and_each_other_bitwise(abp, oracle_states, mode):
    w = wide_batch(*MODES[mode])
    runs = {}
    for sched in (1, 2):
        for ppt in (1, 2, 4):
            res, st, tiles, tun = run(abp, w, particles_per_thread=ppt, schedule=sched)
            assert tun["schedule"] == sched and tun["particles_per_thread"] == ppt
            assert tiles["tiles"] == N_SETS * max(1, M // (256 * ppt)) and tiles["packed"] == 0
            assert tiles["tiles"] >= 152
            assert tiles["narrow"] == 0, (sched, ppt, tiles)  # the wide kernels, not the narrow scalar launch
            runs[(sched, ppt)] = (res, st)
    ref_res, ref_st = runs[(1, 2)]
    # every trajectory against the FP64 oracle
    st = {k: v.cpu().numpy() for k, v in ref_st.items()}
    assert_trajectories_match_oracle(w, st, oracle_states(mode))
    # all six launch forms: the same state and histogram bits
    for key, (res, s) in runs.items():
        for k in ref_st:
            assert torch.equal(s[k], ref_st[k]), (key, k)
        for k in ("hist_x", "hist_v"):
            assert torch.equal(res[k], ref_res[k]), (key, k)
    # equal tiles, equal fixed-order sums: the moments of the two schedules are the same bits
    for ppt in (1, 2, 4):
        assert torch.equal(runs[(1, ppt)][0]["moments"], runs[(2, ppt)][0]["moments"]), ppt
    # histogram rows are complete for every snapshot a set reaches
    hx = ref_res["hist_x"].cpu().numpy()
    for i in range(w.n_sets):
        for k in range(hx.shape[0]):
            assert hx[k, i].sum() == (M if (k + 1) * w.snapshot_every <= w.n_steps[i] else 0)


def test_wide_split_launches_and_graph_replay_are_bitwise(abp):
    # the wide PPT-2 lockstep kernel over windows of 97 steps (unaligned with the 4-step noise
    # blocks and the 64-step folds), run twice so the second run replays captured graphs
    w = wide_batch()
    ref_res, ref_st, _, _ = run(abp, w, particles_per_thread=2, schedule=1)
    with abp.Ensemble(w, particles_per_thread=2, schedule=1, steps_per_launch=97,
                      stream=torch.cuda.Stream()) as ens:
        ens.set_params()
        for rep in range(2):
            if rep:
                ens.reset(w.seed)
            ens.integrate(-1)
            res, st = ens.results(), ens.state()
            torch.cuda.synchronize()
            assert ens.tiles()["narrow"] == 0
            for k in ref_st:
                assert torch.equal(st[k], ref_st[k]), k
            for k in ref_res:
                assert torch.equal(res[k], ref_res[k]), k
