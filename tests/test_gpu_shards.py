"""Sharding on one GPU: an ensemble split into contiguous trajectory ranges, each run by its
own context with abp_config.traj_base = the global id of its first trajectory (as one rank
per GPU would), must give every trajectory bitwise the state of the unsharded run, and the
per-set sums combined across shards (abp_combine_moments) the unsharded moments up to the
order of the FP64 additions.  The weak-scaling replicas of the benchmark are the same construction
(replica r = trajectories [r T, (r + 1) T) of a larger ensemble)."""
import numpy as np
import pytest

from paper_1104_2499_gb300 import shard
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


def batch(M):
    sets = [W._with(D=0.1), W._with(D=0.3, q=2.0, asym=0.1), W._with(D=0.05, F0=0.2)]
    return W.Workload(name="shards", sets=sets, n_traj=[M] * 3, n_steps=[1500, 1500, 1500], dt=1e-3, seed=17,
                      v0_mode=1)


@pytest.mark.parametrize("world", [2, 4])
def test_shards_reproduce_the_unsharded_run(abp, world):
    # one set per shard group: shard r holds trajectories [r m, (r + 1) m) of every set; a
    # one-set workload keeps the global ids of a set contiguous across shards
    m = 1024
    for s in range(3):
        full = batch(m * world)
        one = W.Workload(name="one", sets=[full.sets[s]], n_traj=[m * world], n_steps=[full.n_steps[s]], dt=full.dt,
                         seed=full.seed, v0_mode=full.v0_mode)
        with abp.Ensemble(one) as ens:
            ens.run()
            ref_state = ens.state()
            ref_mom = ens.results(host=True)["moments"].numpy()
        sums = np.zeros((1, 4))
        for r in range(world):
            part = W.Workload(name="part", sets=[full.sets[s]], n_traj=[m], n_steps=[full.n_steps[s]], dt=full.dt,
                              seed=full.seed, v0_mode=full.v0_mode)
            with abp.Ensemble(part, traj_base=r * m) as ens:
                ens.run()
                st = ens.state()
                sums += ens.results(host=True)["moments"].numpy()[:, 4:8]
            for k in st:
                assert torch.equal(st[k], ref_state[k][r * m:(r + 1) * m]), (s, r, k)
        got = np.zeros((1, 8))
        got[0, 4:] = sums
        abp.abp_combine_moments(got, [m * world], [full.n_steps[s]], full.dt)
        np.testing.assert_allclose(got[0, :4], ref_mom[0, :4], rtol=1e-12, atol=1e-15)
        # the same sums combined on the device give the same bits as on the host
        dev = torch.from_numpy(got.copy()).cuda()
        dev[:, :4] = float("nan")
        abp.abp_combine_moments(dev, [m * world], [full.n_steps[s]], full.dt)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), got)


def test_combining_one_shard_reproduces_its_reduction_bitwise(abp):
    # abp_combine_moments applies the reduction's own formulas: one shard's sums give back
    # abp_reduce's derived moments exactly, on the device and on the host
    w = batch(700)
    w.n_steps = [1500, 0, 333]
    with abp.Ensemble(w) as ens:
        ens.run()
        ref = ens.results()["moments"]
        torch.cuda.synchronize()
    dev = ref.clone()
    dev[:, :4] = -1.0
    abp.abp_combine_moments(dev, w.n_traj, w.n_steps, w.dt)
    torch.cuda.synchronize()
    assert torch.equal(dev, ref)
    host = ref.cpu().numpy().copy()
    host[:, :4] = -1.0
    abp.abp_combine_moments(host, w.n_traj, w.n_steps, w.dt)
    assert np.array_equal(host, ref.cpu().numpy())


def test_replica_ids_follow_the_rank(abp):
    # replica r of a batch of T trajectories = trajectories [r T, (r + 1) T) of the batch
    # repeated; its first set's first trajectory is global id r T
    w = batch(64)
    T = w.total_traj
    with abp.Ensemble(w, traj_base=shard.replica_traj_base(1, T)) as ens:
        ens.run()
        rep = ens.state()
    twice = W.Workload(name="twice", sets=w.sets + w.sets, n_traj=w.n_traj * 2, n_steps=w.n_steps * 2, dt=w.dt,
                       seed=w.seed, v0_mode=w.v0_mode)
    with abp.Ensemble(twice) as ens:
        ens.run()
        ref = ens.state()
    for k in rep:
        assert torch.equal(rep[k], ref[k][T:]), k


def test_combining_many_sets_on_the_device(abp):
    # the device form takes the sets in launches of 128: 300 sets, random sums and sizes (zero
    # trajectories, one, zero steps included), bitwise the host form
    rng = np.random.default_rng(5)
    n = 300
    m = np.zeros((n, 8))
    m[:, 4] = rng.normal(size=n)
    m[:, 5] = m[:, 4] ** 2 + rng.uniform(0, 1, n)
    m[:, 6] = rng.normal(size=n)
    m[:, 7] = m[:, 6] ** 2 + rng.uniform(0, 1, n)
    M = rng.integers(0, 5000, n)
    M[:3] = [0, 1, 2]
    N = rng.integers(0, 10 ** 5, n)
    N[3] = 0
    host = m.copy()
    abp.abp_combine_moments(host, M.tolist(), N.tolist(), 1e-3)
    dev = torch.from_numpy(m).cuda()
    abp.abp_combine_moments(dev, M.tolist(), N.tolist(), 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)
    assert np.all(host[0, :4] == 0) and host[1, 1] == 0.0 and host[3, 3] == 0.0
