"""The benchmark's workload -- the D x q sweep, 2,048 sets x 1,024 trajectories (2,097,152) -- in
the benchmark's launch configuration (lockstep, two trajectories per thread, 4,096 tiles: the
wide paired kernel), checked trajectory by trajectory on a sample the oracle recomputes one by
one (the same global ids, so the same noise).  The first 10^3 steps of Sec. 2's model: over them
the FP32 and FP64 paths stay together, so the comparison is deterministic.

Bar (the reading of the per-trajectory tolerance used for the wide-batch test):
|gpu - oracle| <= 1e-4 max(|oracle|, s) + 3 |oracle' - oracle|, s = L for x, the larger of
sqrt(D / gamma0) and v* = sqrt(q / gamma0 - c / d) for v, q / c for e; oracle' = the oracle with
every noise increment larger by 1e-6 relative (D -> D (1 + 2e-6)), the accuracy of the FP32
Box-Muller transform.  At least 99.9% of the sampled trajectories also meet the plain bar.
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


def test_full_sweep_sampled_trajectories_in_the_bench_configuration(abp):
    w = W.sweep_grid(n_steps=1000)
    with abp.Ensemble(w, particles_per_thread=2, schedule=1) as ens:
        ens.run()
        tiles, tun = ens.tiles(), ens.tuning()
        st = {k: v.cpu().numpy() for k, v in ens.state().items()}
    assert tiles["tiles"] == 4096 and tiles["narrow"] == 0 and tun["particles_per_thread"] == 2
    base = w.traj_base()
    rng = np.random.default_rng(2048)
    sets = np.arange(0, w.n_sets, 3)  # 683 sets across the whole D x q grid
    plain_ok = total = 0
    for i in sets:
        p = w.sets[i]
        for t in rng.choice(w.n_traj[i], 2, replace=False):
            gid = base[i] + int(t)
            kw = dict(seed=w.seed, dt=w.dt, n_traj=1, n_steps=w.n_steps[i], traj_base=gid, v0_mode=w.v0_mode,
                      want_states=True)
            r = O.run_set(p, **kw)
            rp = O.run_set(dict(p, D=p["D"] * (1.0 + 2e-6)), **kw)
            vs = max(math.sqrt(p["D"] / p["gamma0"]), math.sqrt(max(p["q"] / p["gamma0"] - p["c"] / p["d"], 0.0)))
            ok = True
            for key, s in (("x", p["L"]), ("x0", p["L"]), ("v", vs), ("e", p["q"] / p["c"])):
                err = abs(st[key][gid] - r[key][0])
                bar = 1e-4 * max(abs(r[key][0]), s)
                assert err <= bar + 3.0 * abs(rp[key][0] - r[key][0]), (int(i), gid, key, err, bar)
                ok &= err <= bar
            plain_ok += ok
            total += 1
    assert plain_ok >= 0.999 * total, (plain_ok, total)
