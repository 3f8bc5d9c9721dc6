"""The checked build (ABP_DEBUG_CHECKS=1), the stand-in for a memory checker: every kernel
checks its tile, set, trajectory, snapshot, checkpoint and sub-checkpoint indices before the
access and records status 3 (reported as ABP_ESTATE) on a violation.

Bar: a child process runs the same workloads against the release and the checked library --
ragged batches with one-set and packed tiles, snapshots and split launches under both
schedules, stochastic Heun, xorshift noise, warp-specialised narrow launches (one set of 32-wide
blocks, and 16,384 packed work items planned 64 wide and split into 32-thread blocks), the full and
windowed adjoint with its per-trajectory readout (with and without the hand-off of Philox blocks
from level 1 to the reverse sweep), and the combination of moments on the device --
and no check may fail, and every state, result and gradient must be the
release library's bits (the checks change no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
import numpy as np
sys.path.insert(0, os.environ["ABP_ROOT"])
from paper_1104_2499_gb300 import abp as A, workloads as W

out = {}
sets = [W.params(D=0.1), W.params(D=0.5, q=3.0, asym=0.0), W.params(D=0.02, q=0.3, gamma0=2.0, F0=0.2),
        W.params(D=0.3, L=2.0, h=0.5, asym=0.4)] + [W.params(D=0.05 + 0.01 * i) for i in range(20)]


def ragged(**kw):
    return W.Workload(name="ragged", sets=sets, n_traj=[300, 1, 1025, 513] + [3] * 20,
                      n_steps=[700, 697, 10, 700] + [700] * 20, dt=1e-3, seed=41, v0_mode=1, hist_x_bins=16,
                      hist_v_bins=8, v_lo=-2.0, v_hi=2.0, snapshot_every=97, **kw)


runs = [("lockstep", ragged(), dict(schedule=1, particles_per_thread=2, steps_per_launch=53)),
        ("queue", ragged(), dict(schedule=2, particles_per_thread=2)),
        ("heun", ragged(scheme=1), dict(schedule=1, particles_per_thread=2)),
        ("xorshift", ragged(noise=1), dict(schedule=1, particles_per_thread=1)),
        ("narrow", W.single_set(n_traj=4096, n_steps=1003, hist_x_bins=32),
         dict(schedule=1, particles_per_thread=1, steps_per_launch=250)),
        ("narrow64", W.force_sweep(n_F=16384, traj_per_set=1, n_steps=300),
         dict(schedule=1, particles_per_thread=1, steps_per_launch=130))]
for tag, w, kw in runs:
    with A.Ensemble(w, **kw) as ens:
        ens.run()
        ens.synchronize()
        for k, v in ens.state().items():
            out["%s/state/%s" % (tag, k)] = v.cpu().numpy()
        for k, v in ens.results().items():
            if v is not None:
                out["%s/results/%s" % (tag, k)] = v.cpu().numpy()
w = W.Workload(name="adj", sets=sets[:3], n_traj=[256, 100, 300], n_steps=[2000, 1900, 777], dt=1e-3, seed=31,
               v0_mode=1, checkpoint_every=333)
with A.Ensemble(w, schedule=1, particles_per_thread=2) as ens:
    ens.run()
    out["adjoint/grad"] = ens.backward(host=True).numpy()
    out["adjoint/windowed"] = ens.backward(host=True, window=666).numpy()
    out["adjoint/traj"] = ens.traj_grad(host=True).numpy()
    ens.synchronize()
w.checkpoint_every = 256  # whole 8-step sub-chunks: level 1 hands its Philox blocks to the reverse sweep
with A.Ensemble(w, schedule=1, particles_per_thread=2) as ens:
    ens.run()
    out["adjoint256/grad"] = ens.backward(host=True).numpy()
    out["adjoint256/windowed"] = ens.backward(host=True, window=512).numpy()
    out["adjoint256/traj"] = ens.traj_grad(host=True).numpy()
    ens.synchronize()
w.checkpoint_every = 500
with A.Ensemble(w, schedule=1, particles_per_thread=2) as ens:
    ens.run()
    out["adjoint500/grad"] = ens.backward(host=True).numpy()
    out["adjoint500/traj"] = ens.traj_grad(host=True).numpy()
    mom = ens.results()["moments"]
    mom[:, :4] = 0.0
    A.abp_combine_moments(mom, w.n_traj, w.n_steps, w.dt)
    ens.synchronize()
    out["combine"] = mom.cpu().numpy()
np.savez(sys.argv[1], **out)
'''


def test_checked_build_runs_clean_and_gives_the_release_bits(tmp_path):
    from paper_1104_2499_gb300 import build as B

    libs = {"release": B.build(), "checked": B.build(extra=["-DABP_DEBUG_CHECKS=1"], out_dir=B.CHECKED_OUT)}
    outs = {}
    for name, lib in libs.items():
        path = str(tmp_path / (name + ".npz"))
        env = dict(os.environ, ABP_LIB=lib, ABP_ROOT=ROOT)
        r = subprocess.run([sys.executable, "-c", CHILD, path], env=env, capture_output=True, text=True,
                           timeout=900, cwd=ROOT)
        assert r.returncode == 0, (name, r.stderr[-4000:])
        outs[name] = np.load(path)
    assert sorted(outs["release"].files) == sorted(outs["checked"].files)
    for k in outs["release"].files:
        np.testing.assert_array_equal(outs["release"][k], outs["checked"][k], err_msg=k)
