"""Host-side checkpoint / resume (abp_save, abp_load): an interrupted run resumed from an
image, in a fresh context, gives bitwise the results of an uninterrupted run."""
import numpy as np
import pytest

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


def batch():
    sets = [W._with(D=0.1), W._with(D=0.4, q=2.0, asym=0.1), W._with(D=0.02, F0=0.1)]
    return W.Workload(name="resume", sets=sets, n_traj=[700, 33, 300], n_steps=[900, 451, 900], dt=1e-3, seed=77,
                      v0_mode=1, hist_x_bins=24, hist_v_bins=12, v_lo=-2.0, v_hi=2.0, snapshot_every=150)


@pytest.mark.parametrize("device_image", [False, True])
def test_resume_is_bitwise_identical(abp, device_image):
    w = batch()
    with abp.Ensemble(w) as ref:
        ref.run()
        r_ref, s_ref = ref.results(), ref.state()
    with abp.Ensemble(w) as a:
        a.set_params()
        a.integrate(301)
        img = abp.abp_save(a.ctx) if not device_image else None
        if device_image:
            n = abp.abp_save(a.ctx).nbytes
            img = torch.empty(n, dtype=torch.uint8, device="cuda")
            abp.abp_save(a.ctx, img)
    with abp.Ensemble(w) as b:  # a fresh context
        b.set_params()
        b.integrate(50)  # state to be overwritten
        abp.abp_load(b.ctx, img)
        assert abp.abp_progress(b.ctx, w.n_sets) == [301, 301, 301]
        b.integrate(-1)
        r_b, s_b = b.results(), b.state()
    for k in s_ref:
        assert torch.equal(s_ref[k], s_b[k]), k
    for k in r_ref:
        assert torch.equal(r_ref[k], r_b[k]), k


def test_load_rejects_other_batches_and_blocks_backward(abp):
    w = batch()
    w.checkpoint_every = 100
    with abp.Ensemble(w) as a:
        a.set_params()
        a.integrate(200)
        img = abp.abp_save(a.ctx)
    other = batch()
    other.n_traj = [701, 33, 300]
    with abp.Ensemble(other) as b:
        b.set_params()
        with pytest.raises(abp.AbpError) as ei:
            abp.abp_load(b.ctx, img)
        assert ei.value.status == abp.ABP_EINVAL
    with abp.Ensemble(w) as c:
        c.set_params()
        abp.abp_load(c.ctx, img)
        c.integrate(-1)
        with pytest.raises(abp.AbpError) as ei:
            c.backward()
        assert ei.value.status == abp.ABP_ESTATE
        bad = img.copy()
        bad[:8] = 0
        with pytest.raises(abp.AbpError):
            abp.abp_load(c.ctx, bad)
