"""Host-side checks of the allocation-free entry point's Python wrapper (no GPU needed).

The C entry point cannot see the extent of the caller's output buffers, so the wrapper
checks their type, size and device before the call: an undersized or mistyped buffer
would otherwise be written past its end by the device."""
import pytest

torch = pytest.importorskip("torch")

from paper_1104_2499_gb300 import abp as A
from paper_1104_2499_gb300 import workloads as W


def _cfg(**kw):
    w = W.Workload(name="w", sets=[W._with()], n_traj=[100], n_steps=[1000], dt=1e-3, seed=1, hist_x_bins=16,
                   hist_v_bins=8, snapshot_every=250, **kw)
    return w, A.make_config(w)


def test_snapshot_rows():
    w, cfg = _cfg()
    assert A.noalloc_snapshots(cfg, 1000) == 4 and A.noalloc_snapshots(cfg, 999) == 3
    cfg.snapshot_every = 0
    assert A.noalloc_snapshots(cfg, 1000) == 1
    cfg.hist_x_bins = cfg.hist_v_bins = 0
    assert A.noalloc_snapshots(cfg, 1000) == 0


def test_wrapper_rejects_bad_outputs_before_calling_the_library():
    w, cfg = _cfg()
    good = dict(moments=torch.zeros(8, dtype=torch.float64), hist_x=torch.zeros((4, 16), dtype=torch.int32),
                hist_v=torch.zeros((4, 10), dtype=torch.int32))
    bad = [
        dict(moments=torch.zeros(7, dtype=torch.float64)),          # too small
        dict(moments=torch.zeros(8, dtype=torch.float32)),          # wrong type
        dict(hist_x=torch.zeros((3, 16), dtype=torch.int32)),       # one snapshot short
        dict(hist_x=None),                                          # required: hist_x_bins > 0
        dict(hist_v=torch.zeros((4, 9), dtype=torch.int32)),        # the two out-of-range counters missing
        dict(hist_v=torch.zeros((4, 10), dtype=torch.int64)),       # 8-byte counts
        {},                                                         # right sizes, but host memory
    ]
    for b in bad:
        kw = dict(good, **b)
        with pytest.raises(ValueError):
            A.abp_run_set_noalloc(w.sets[0], cfg, 100, 1000, kw["moments"], kw["hist_x"], kw["hist_v"])
