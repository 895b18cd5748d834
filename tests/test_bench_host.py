"""Host-side logic of bench.py (no GPU): the per-call pass counts behind
`gpu_launches` and the e2e byte accounting, the start-node sample, and the
cost-balanced shard cuts."""
import numpy as np

import bench
import synth
import paper_2404_11105_b300 as xm


def test_passes_per_call():
    # one matching pass, or one per split part and quotient plus the product kernel
    assert bench.passes_per_call(xm.Plan(synth.CYCLE4), True) == (1, 0)
    assert bench.passes_per_call(xm.Plan(synth.BIPARALLEL), False) == (1, 0)
    ff = xm.Plan(synth.FFCHAIN5)
    sp = ff.split()
    assert bench.passes_per_call(ff, True) == (len(sp["parts"]) + len(sp["quotients"]), 1) == (5, 1)
    assert bench.passes_per_call(ff, False) == (5, 1)
    # a split whose cut vertex is not the start vertex walks over subsets
    path5 = xm.Plan((5, [(0, 1), (1, 2), (2, 3), (3, 4)]))
    assert path5.split()["cut"] >= 0 and "start-node subsets walked" in path5.describe()
    assert bench.passes_per_call(path5, True) == (1, 0)
    assert bench.passes_per_call(path5, False)[1] == 1


def test_start_node_sample_is_seeded_sorted_and_distinct():
    a, desc = bench.start_node_sample(1 << 16, 64)
    b, _ = bench.start_node_sample(1 << 16, 64)
    assert np.array_equal(a, b) and len(a) == 1024 and "1/64" in desc
    assert np.all(np.diff(a) > 0) and a.min() >= 0 and a.max() < (1 << 16)


def test_balanced_cuts_split_cost_evenly():
    rng = np.random.default_rng(3)
    cost = rng.pareto(1.2, 5000) + 1.0
    for world in (1, 2, 3, 8):
        cuts = bench.balanced_cuts(cost, world)
        assert cuts[0] == 0 and cuts[-1] == len(cost) and len(cuts) == world + 1
        assert all(a <= b for a, b in zip(cuts, cuts[1:]))
        shares = [cost[a:b].sum() for a, b in zip(cuts, cuts[1:])]
        # every shard within one heaviest node of the even share
        assert max(shares) <= cost.sum() / world + cost.max() + 1e-9


def test_plan_bytes_match_the_device_plan_layout():
    # XmPlanDev: k, order[8], four product words, then 8 levels and 7 product
    # sets; a device level is the ABI's xm_level_info without its `vertex`
    import ctypes
    level = ctypes.sizeof(xm.xm_level_info) - 4
    assert level == 260
    assert bench.PLAN_BYTES == 4 + 4 * 8 + 4 * 4 + 15 * level
