"""Batched matching: every (pattern, graph) pair's count from one launch
equals xm_count on that pair and the oracle; tunings, CUDA-graph replay and
the autotuner do not change results."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xm():
    import paper_2404_11105_b300 as m
    return m


@pytest.fixture(scope="module")
def setup(xm):
    graphs = [synth.small_graph(i, seed=41, n_lo=20, n_hi=300) for i in range(10)]
    # named patterns, leaf-product patterns (choose and inclusion-exclusion
    # forms: the batched walk ends in the product), random ones
    pats = [synth.CYCLE3, synth.FFL, synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5, (2, [(0, 1)])] + \
           [synth.LEAF_PRODUCT_PATTERNS[k] for k in ("out_star4", "path4", "out_star5")] + \
           [synth.batch_pattern(i, seed=43, k_hi=5) for i in range(6)]
    xg = [xm.Graph(*g) for g in graphs]
    og = [oracle.OracleGraph(*g) for g in graphs]
    xp = [xm.Plan(p) for p in pats]
    pairs = [(pi, gi) for pi in range(len(pats)) for gi in range(len(graphs))]
    return pats, xg, og, xp, pairs


def test_batch_equals_single_and_oracle(xm, setup):
    pats, xg, og, xp, pairs = setup
    counts = xm.xm_count_batch(xp, xg, pairs)
    for (pi, gi), c in zip(pairs, counts):
        assert c == xm.xm_count(xg[gi], xp[pi]), (pi, gi)
    # oracle on a subset of pairs (all patterns, first three graphs)
    for (pi, gi), c in zip(pairs, counts):
        if gi < 3:
            assert c == og[gi].count_matches(pats[pi]), (pi, gi)


def test_batch_tunings_graph_replay_and_autotuner(xm, setup):
    pats, xg, og, xp, pairs = setup
    ref = xm.xm_count_batch(xp, xg, pairs)
    b = xm.Batch(xp, xg, pairs)
    for t in (dict(window=64, unit=1, warps_per_block=2), dict(window=96, unit=7), dict(window=512, unit=128)):
        b.set_tuning(**t)
        b.run()
        assert b.counts() == ref, t
    # captured CUDA graph, replayed twice
    b.run(graph=True)
    assert b.counts() == ref
    b.run(graph=True)
    assert b.counts() == ref
    best, ms = b.tune([(128, 16, 4, 0, 0), (256, 64, 8, 0, 0), (64, 4, 8, 2, 0)], reps=2)
    launch = {k: best[k] for k in ("window", "unit", "warps_per_block", "blocks_per_sm", "budget_ms")}
    assert ms > 0 and best["merge_ratio"] == 2 and launch in (
        {"window": 128, "unit": 16, "warps_per_block": 4, "blocks_per_sm": 0, "budget_ms": 0},
        {"window": 256, "unit": 64, "warps_per_block": 8, "blocks_per_sm": 0, "budget_ms": 0},
        {"window": 64, "unit": 4, "warps_per_block": 8, "blocks_per_sm": 2, "budget_ms": 0})
    b.run()
    assert b.counts() == ref
    b.free()


def test_batch_rejects_bad_pairs(xm, setup):
    pats, xg, og, xp, pairs = setup
    with pytest.raises(xm.XmError):
        xm.Batch(xp, xg, [(0, len(xg))])


def test_batch_per_pair_budget(xm, setup):
    """With a per-pair budget, a pair that needs far more than its budget is
    reported as timed out while every other pair of the same launch keeps
    its exact count; without a budget every pair reports XM_OK."""
    pats, xg, og, xp, pairs = setup
    n, src, dst = synth.rmat_graph(14, 16, seed=5)
    heavy_g = xm.Graph(n, src, dst)
    # a directed 6-cycle: no leaf product and no cut vertex, so the batch
    # walks all six levels; below the hubs that takes seconds at least
    heavy_p = xm.Plan((6, [(i, (i + 1) % 6) for i in range(6)]))
    assert heavy_p.product()["r"] == 0
    graphs = xg + [heavy_g]
    plans = xp + [heavy_p]
    heavy = (len(plans) - 1, len(graphs) - 1)
    # heavy pairs before and after the light ones: light units queued behind
    # heavy units in a warp's grab are not charged for the wait
    # light pairs: the patterns of at most four vertices (a five-vertex walk
    # on these graphs can itself take a second per unit)
    light_pairs = [(pi, gi) for pi, gi in pairs if pats[pi][0] <= 4]
    hp = [heavy] + light_pairs + [heavy]
    want = xm.xm_count_batch(xp, xg, light_pairs)
    b = xm.Batch(plans, graphs, hp)
    # wall-clock budget: light units share the SMs with heavy units, so the
    # budget sits far above a light unit's time under that contention
    b.set_pair_budget(200)
    b.run()
    counts = b.counts()
    st = b.pair_status()
    assert st[0] == xm.XM_ETIMEOUT and st[-1] == xm.XM_ETIMEOUT
    assert (st[1:-1] == xm.XM_OK).all(), np.nonzero(st[1:-1])
    assert counts[1:-1] == want
    b.free()
    light = xm.Batch(xp, xg, light_pairs)
    light.set_pair_budget(0)
    light.run()
    assert (light.pair_status() == xm.XM_OK).all() and light.counts() == want
    light.free()
