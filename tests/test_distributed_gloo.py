"""Multi-process ensemble on CPU ranks (gloo, world size 2).

Each rank integrates its replica of a batch with the FP64 oracle (trajectory ids offset by
rank, as abp_config.traj_base does on the GPU), the per-set sums are all-reduced and the
library's abp_combine_moments (host memory: no GPU needed) forms the moments of the combined
ensemble on every rank; they must equal those of the concatenated ensemble computed in one
process from the per-trajectory values.
Failure detection is tested on the host: a rank that leaves before the collective makes the
other rank's all-reduce fail after its timeout instead of hanging.
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from paper_1104_2499_gb300 import shard
from paper_1104_2499_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1104_2499_gb300 import build as B

    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available to build libabp.so")
    return B.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _batch():
    sets = [W._with(D=0.1), W._with(D=0.3, q=2.0, asym=0.1)]
    return W.Workload(name="gloo", sets=sets, n_traj=[40, 25], n_steps=[600, 600], dt=1e-3, seed=5, v0_mode=1)


def _oracle_local(w, traj_base):
    import sys

    sys.path.insert(0, ROOT)
    from oracle import oracle as O

    mom = np.zeros((w.n_sets, 8))
    per = []
    for i, p in enumerate(w.sets):
        r = O.run_set(p, seed=w.seed, dt=w.dt, n_traj=w.n_traj[i], n_steps=w.n_steps[i],
                      traj_base=traj_base + w.traj_base()[i], v0_mode=w.v0_mode, want_states=True, n_threads=1)
        mom[i, 4:] = r["sums"]
        per.append((r["vbar"], r["x"] - r["x0"]))
    return mom, per


def _worker(rank, world, port, out_dir, fail_rank):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    w = _batch()
    local, _ = _oracle_local(w, shard.replica_traj_base(rank, w.total_traj))
    if rank == fail_rank:
        os._exit(0)  # leaves without joining the collective (host-side failure)

    def all_reduce(a):
        t = torch.from_numpy(a)
        dist.all_reduce(t)
        return t.numpy()

    status = "ok"
    try:
        res = shard.combine(local, w.n_traj, w.n_steps, w.dt, world, all_reduce)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank), res)
        # the benchmark's in-place form on a torch moments tensor (a strided column view):
        # every column, the derived moments included, is that of the combined ensemble
        mom = torch.from_numpy(local.copy())
        shard.all_reduce_sums_(mom, dist.all_reduce, [m * world for m in w.n_traj], w.n_steps, w.dt)
        np.testing.assert_array_equal(mom.numpy(), res)
    except Exception as e:  # the collective ended with an error instead of hanging
        status = "error: " + type(e).__name__
    with open(os.path.join(out_dir, "status%d.txt" % rank), "w") as f:
        f.write(status)
    if status == "ok":
        dist.destroy_process_group()


def _run(world, fail_rank, tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path), fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank did not finish")
    return procs


def test_replicas_combine_to_the_concatenated_ensemble(tmp_path):
    procs = _run(2, -1, tmp_path)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        assert (tmp_path / ("status%d.txt" % r)).read_text() == "ok"
    w = _batch()
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    np.testing.assert_array_equal(r0, r1)
    # one process, both replicas, per-trajectory values concatenated
    per = [_oracle_local(w, shard.replica_traj_base(r, w.total_traj))[1] for r in range(2)]
    for i in range(w.n_sets):
        vbar = np.concatenate([per[r][i][0] for r in range(2)])
        dx = np.concatenate([per[r][i][1] for r in range(2)])
        M = vbar.size
        assert r0[i, 0] == pytest.approx(vbar.mean(), rel=1e-12)
        assert r0[i, 1] == pytest.approx(vbar.std(ddof=1) / np.sqrt(M), rel=1e-9)
        assert r0[i, 2] == pytest.approx(np.mean(dx ** 2), rel=1e-12)
        T = w.n_steps[i] * w.dt
        assert r0[i, 3] == pytest.approx(dx.var() / (2 * T), rel=1e-9)


def test_a_rank_that_leaves_makes_the_collective_fail_not_hang(tmp_path):
    procs = _run(2, 1, tmp_path)
    status = (tmp_path / "status0.txt").read_text()
    assert status.startswith("error"), status
    assert not (tmp_path / "status1.txt").exists()


def test_combined_moments_edge_cases():
    from paper_1104_2499_gb300 import abp as A

    # an empty set has no moments; one trajectory has no standard error; zero steps no D_eff
    m = np.zeros((3, 8))
    m[1, 4:] = [2.0, 4.0, 4.0, 16.0]  # one trajectory: vbar = 2, dx = 4
    m[2, 4:] = [2.0, 2.0, 4.0, 8.0]  # two trajectories, vbar = 1 each, dx = 2 each
    A.abp_combine_moments(m, [0, 1, 2], [100, 2000, 0], 1e-3)
    assert np.all(m[0] == 0)
    assert m[1].tolist() == [2.0, 0.0, 16.0, 0.0, 2.0, 4.0, 4.0, 16.0]
    assert m[2, :4].tolist() == [1.0, 0.0, 4.0, 0.0]
    # the sample variance of (a, b) is (a - b)^2 / 2, the standard error |a - b| / 2
    a, b, dxa, dxb = 0.3, -0.1, 0.6, -0.2
    m = np.zeros((1, 8))
    m[0, 4:] = [a + b, a * a + b * b, dxa + dxb, dxa * dxa + dxb * dxb]
    A.abp_combine_moments(m, [2], [2000], 1e-3)
    assert m[0, 0] == pytest.approx((a + b) / 2, rel=1e-15)
    assert m[0, 1] == pytest.approx(abs(a - b) / 2, rel=1e-12)
    assert m[0, 3] == pytest.approx(((dxa - dxb) / 2) ** 2 / (2 * 2.0), rel=1e-12)
    with pytest.raises(A.AbpError):
        A.abp_combine_moments(np.zeros((1, 8)), [-1], [10], 1e-3)
    with pytest.raises(A.AbpError):
        A.abp_combine_moments(np.zeros((1, 8)), [1], [10], 0.0)
    with pytest.raises(ValueError):
        A.abp_combine_moments(np.zeros((1, 4)), [1], [10], 1e-3)
