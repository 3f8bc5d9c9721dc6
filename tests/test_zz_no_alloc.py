"""The allocation-free entry point (abp_run_set_noalloc) against the context entry points.

Callers that cannot allocate device memory (a host framework that owns all device memory
through its own pool, a loop that must not stall on cudaMalloc) use abp_run_set_noalloc,
whose scratch is a static device array.  It must give the same moments and histograms as
abp_set_params + abp_integrate + abp_reduce for the same set, on consecutive calls that
reuse the shared scratch.  Collected last on purpose (file name) so that a failure here
does not hide the other tests in a run that stops at the first failure.
"""
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


def _reference(A, w):
    with A.Ensemble(w) as ens:
        ens.run()
        res = ens.results()
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in res.items()}


def _noalloc(A, w):
    cfg = A.make_config(w)
    ns = (w.n_steps[0] // w.snapshot_every) if w.snapshot_every > 0 else 1
    mom = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    hx = torch.full((ns, w.hist_x_bins), -1, dtype=torch.int32, device="cuda")
    hv = torch.full((ns, w.hist_v_bins + 2), -1, dtype=torch.int32, device="cuda")
    A.abp_run_set_noalloc(w.sets[0], cfg, w.n_traj[0], w.n_steps[0], mom, hx, hv)
    torch.cuda.synchronize()
    return mom, hx, hv


def test_noalloc_matches_context_entry_points_on_consecutive_calls(abp):
    cases = [
        W.Workload(name="na1", sets=[W._with(D=0.1)], n_traj=[3001], n_steps=[1500], dt=1e-3, seed=41, v0_mode=1,
                   hist_x_bins=64, hist_v_bins=30, v_lo=-3.0, v_hi=3.0, snapshot_every=500),
        W.Workload(name="na2", sets=[W._with(D=0.4, q=2.5, asym=0.1)], n_traj=[777], n_steps=[1203], dt=1e-3,
                   seed=42, v0_mode=0, hist_x_bins=32, hist_v_bins=10, v_lo=-2.0, v_hi=2.0, snapshot_every=400),
    ]
    for w in cases:  # two calls in a row share (and reuse) the static scratch
        ref = _reference(abp, w)
        mom, hx, hv = _noalloc(abp, w)
        # same kernels, same arithmetic: agreement far inside the 3-SE / 1e-4 bars of the
        # oracle comparisons; the histograms are integer counts and must be equal
        np.testing.assert_allclose(mom.cpu().numpy(), ref["moments"][0].cpu().numpy(), rtol=1e-12, atol=1e-15)
        assert torch.equal(hx, ref["hist_x"][:, 0, :])
        assert torch.equal(hv, ref["hist_v"][:, 0, :])
        assert int(hx[0].sum()) == w.n_traj[0]


def test_noalloc_rejects_ensembles_beyond_the_static_scratch(abp):
    w = W.single_set(n_traj=10, n_steps=10)
    cfg = abp.make_config(w)
    mom = torch.empty(8, dtype=torch.float64, device="cuda")
    hx = torch.empty((1, w.hist_x_bins), dtype=torch.int32, device="cuda")
    with pytest.raises(abp.AbpError) as ei:
        abp.abp_run_set_noalloc(w.sets[0], cfg, 65537, 10, mom, hx)
    assert ei.value.status == abp.ABP_EINVAL and "65536" in str(ei.value)
