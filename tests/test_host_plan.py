"""Host logic of the library on the CPU (no GPU): the tiling abp_set_params applies --
one-set tiles, packed tiles of small sets, narrow launches of small batches -- and the
busy-fraction model the autotuner uses to weigh schedules against a batch."""
import math

import pytest

from paper_1104_2499_gb300 import workloads as W


@pytest.fixture(scope="module")
def A():
    from paper_1104_2499_gb300 import abp
    from paper_1104_2499_gb300 import build as B

    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    B.build()
    abp.lib()
    return abp


def test_one_set_tiles(A):
    p = A.abp_plan([600, 1, 0, 512], [100] * 4, schedule=2, particles_per_thread=2)
    # 512-trajectory tiles, a set never spans two tiles, an empty set has none
    assert p["tile_count"] == [512, 88, 1, 512] and p["tile_set"] == [0, 0, 1, 3]
    assert p["tile_first"] == [0, 512, 600, 601] and p["packed"] == 0 and p["narrow"] == 0


def test_packing_rules(A):
    M = [3, 0, 5, 300, 2, 2, 7, 250, 9]
    N = [100, 100, 100, 100, 100, 100, 50, 50, 50]
    p = A.abp_plan(M, N, schedule=1, particles_per_thread=1, sm_count=4)
    # runs of consecutive small sets (< 256 trajectories, equal step counts, at most 256 in
    # all, at least two non-empty) share a tile: sets 0-2 (3 + 0 + 5) and 4-5 (2 + 2); set 6
    # would reach 257 with set 7, and 7 + 8 would reach 259, so 6, 7 and 8 keep their own tiles
    n_single = p["tiles"] - p["packed"]
    single = list(zip(p["tile_count"], p["tile_set"]))[:n_single]
    packed = list(zip(p["tile_first"], p["tile_count"], p["tile_set"]))[n_single:]
    assert single == [(256, 3), (44, 3), (7, 6), (250, 7), (9, 8)]
    assert packed == [(0, 8, 0), (308, 4, 4)]
    # the work queue and adjoint checkpoints never pack
    assert A.abp_plan(M, N, schedule=2, particles_per_thread=1)["packed"] == 0
    assert A.abp_plan(M, N, schedule=1, particles_per_thread=1, checkpoints=True)["packed"] == 0
    # a lone small set is not packed; a group's lead is its first non-empty set
    assert A.abp_plan([5], [10], schedule=1, particles_per_thread=1)["packed"] == 0
    q = A.abp_plan([0, 4, 6], [10, 10, 10], schedule=1, particles_per_thread=1)
    assert q["packed"] == 1 and q["tile_set"] == [1] and q["tile_first"] == [0] and q["tile_count"] == [10]


def test_narrow_width(A):
    # 4,096 trajectories, PPT 2: 8 tiles < 152 SMs; no width >= 64 gives 152 blocks -> 32
    assert A.abp_plan([4096], [10], 1, 2)["narrow"] == 32
    # 19,456 trajectories, PPT 1: 76 tiles; width 128 gives exactly 152 blocks
    assert A.abp_plan([19456], [10], 1, 1)["narrow"] == 128
    # enough tiles, or the work queue: not narrow
    assert A.abp_plan([152 * 256], [10], 1, 1)["narrow"] == 0
    assert A.abp_plan([4096], [10], 2, 1)["narrow"] == 0


def test_busy_fraction_model(A):
    # whole waves of full tiles: lockstep keeps every unit busy
    assert A.abp_plan_efficiency([456 * 512 * 3], [10_000], 1, 2, units=456) == pytest.approx(1.0)
    # 1.12 waves: the second wave is 12% full
    M = [4096] * 64
    e = A.abp_plan_efficiency(M, [100_000] * 64, 1, 2, units=456)
    assert e == pytest.approx(512 / (2 * 456), rel=1e-9)
    # the work queue spreads the same tiles over all units: equal items of 10^3 steps (the
    # largest size giving 32 per unit), ceil(51,200 / 456) = 113 of them on the busiest unit
    ewq = A.abp_plan_efficiency(M, [100_000] * 64, 2, 2, units=456)
    assert ewq == pytest.approx(51_200 / (113 * 456), rel=1e-12) and ewq > e
    # a single long set bounds the work queue by its chain
    e1 = A.abp_plan_efficiency([256], [1000], 2, 1, units=100)
    assert e1 == pytest.approx(0.01)
    # one-trajectory work items: packed in lockstep (full tiles), one slot in 256 otherwise
    items = A.abp_plan_efficiency([1] * 4096, [1000] * 4096, 1, 1, units=16)
    assert items == pytest.approx(1.0)
    assert A.abp_plan_efficiency([1] * 4096, [1000] * 4096, 2, 1, units=16) < 0.01


def test_trial_batch_busy_fraction(A):
    # the autotuner's trial batch (4,096 trajectories per SM, 8,192 timed steps) against the
    # units it passes, the SMs (one resident block draws an SM's full rate): 16, 8 or 4 tiles
    # per SM, whole waves for lockstep at every PPT, and for the work queue in four rounds of
    # 2,048 steps 4 x 1,216 / 152 = 32 equal items per SM -- no tail anywhere
    T = 152 * 4096
    for ppt in (1, 2, 4):
        assert A.abp_plan_efficiency([T], [8192], 1, ppt, units=152, steps_per_launch=8192) == pytest.approx(1.0)
        assert A.abp_plan_efficiency([T], [8192], 2, ppt, units=152, steps_per_launch=2048) == pytest.approx(1.0)
    # counted in resident blocks instead (3 per SM at PPT 2), the same batch would lose a third
    # of its last wave: 1,216 tiles on 456 blocks, 2.67 waves
    assert A.abp_plan_efficiency([T], [8192], 1, 2, units=456, steps_per_launch=8192) == pytest.approx(
        (1216 / 456) / 3, rel=1e-9)


def test_work_queue_tail_steps_with_whole_items_per_unit(A):
    # equal items (one set, its step count a multiple of the item size): the makespan is
    # ceil(items / units) items -- the staircase measured on GB300 with one to three blocks
    # per SM -- so the busy fraction is items / (units * ceil(items / units))
    for tiles, units in ((4096, 152), (2048, 152), (1824, 152), (1825, 152)):
        M = [tiles * 512]
        e = A.abp_plan_efficiency(M, [3840], 2, 2, units=units, steps_per_launch=3840)
        assert e == pytest.approx(tiles / (units * math.ceil(tiles / units)), rel=1e-12), tiles
    # 26.95 items per SM: 0.2% idle; 13.47: 3.8% idle
    assert A.abp_plan_efficiency([4096 * 512], [3840], 2, 2, units=152, steps_per_launch=3840) > 0.997
    assert A.abp_plan_efficiency([2048 * 1024], [3840], 2, 4, units=152, steps_per_launch=3840) < 0.97


def test_invalid_plans_are_refused(A):
    with pytest.raises(A.AbpError):
        A.abp_plan([10], [10], schedule=3, particles_per_thread=1)
    with pytest.raises(A.AbpError):
        A.abp_plan([10], [10], schedule=1, particles_per_thread=3)
    with pytest.raises(A.AbpError):
        A.abp_plan([-1], [10], schedule=1, particles_per_thread=1)


def test_work_queue_tail_follows_the_item_size(A):
    # unequal tiles (sets of different step counts): the tile-steps spread over the units
    # plus half a work item of tail, at the item size the candidate uses (the autotuner ranks
    # 10^3, 10^4, 10^5), never less than the longest tile
    M, N, units = [4096] * 64, [100_000] * 32 + [50_000] * 32, 152
    tile_steps = 256 * 100_000 + 256 * 50_000  # 64 sets x 8 tiles of 512 trajectories
    useful = 32 * 4096 * 100_000 + 32 * 4096 * 50_000
    for S in (1000, 10_000, 100_000):
        e = A.abp_plan_efficiency(M, N, 2, 2, units=units, steps_per_launch=S)
        span = max(tile_steps / units + 0.5 * S, 100_000)
        assert e == pytest.approx(useful / (units * span * 512), rel=1e-12), S
    e1 = A.abp_plan_efficiency(M, N, 2, 2, units=units, steps_per_launch=1000)
    e5 = A.abp_plan_efficiency(M, N, 2, 2, units=units, steps_per_launch=100_000)
    assert e1 > 0.99 and e5 < 0.9
