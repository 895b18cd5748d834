"""Multi-rank path of bench.py on CPU: world_size-2 gloo ranks each count
their start-node shard (the oracle stands in for a rank's GPU), and the
limb-wise all-reduce recovers the exact whole-graph counts."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

PATTERNS = {"ffl": synth.FFL, "cycle4": synth.CYCLE4, "bifan": synth.BIFAN}


def _graph(kind):
    return synth.er_graph(300, 2400, seed=21) if kind == "er" else synth.rmat_graph(9, 6, seed=23)


def _rank(rank, world, port, q, kind):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, src, dst = _graph(kind)
    og = oracle.OracleGraph(n, src, dst)
    lo, hi = bench.shard_bounds(n, src, dst, world)[rank]
    part = {}
    for name, pat in PATTERNS.items():
        aut = oracle.automorphisms(pat).shape[0]
        part[name] = og.count_embeddings(pat, 0, lo, hi) * (1 << 70) // aut  # large values exercise the limbs
    total = bench.allreduce_counts(part, dist)
    if rank == 0:
        q.put(total)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["er", "rmat"])
def test_two_rank_shards_sum_to_whole(kind):
    import bench
    import oracle
    n, src, dst = _graph(kind)
    b = bench.shard_bounds(n, src, dst, 2)
    assert b[0][0] == 0 and b[-1][1] == n and b[0][1] == b[1][0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() + (7 if kind == "rmat" else 0)) % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, kind)) for r in range(2)]
    for p in procs:
        p.start()
    total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    og = oracle.OracleGraph(n, src, dst)
    for name, pat in PATTERNS.items():
        aut = oracle.automorphisms(pat).shape[0]
        assert total[name] == og.count_embeddings(pat) * (1 << 70) // aut


def test_cost_balanced_shards_on_a_power_law_graph():
    """On an R-MAT graph (hubs at low ids) the cost-balanced ranges give each
    of four ranks a similar share of the estimated walk work, where ranges of
    equal degree sums would leave the first rank with most of it; the same
    holds for pieces of a start-node sample; the pieces cover every node
    once."""
    import bench
    n, src, dst = synth.rmat_graph(12, 8, seed=7)
    cost = bench.root_costs(n, src, dst)
    b = bench.shard_bounds(n, src, dst, 4)
    assert [x for r in b for x in r][::2][0] == 0 and b[-1][1] == n
    assert all(b[r][1] == b[r + 1][0] for r in range(3))
    share = np.array([cost[lo:hi].sum() for lo, hi in b]) / cost.sum()
    deg = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    dcum = np.cumsum(deg)
    dcuts = [0] + [int(np.searchsorted(dcum, dcum[-1] * r / 4)) for r in range(1, 4)] + [n]
    dshare = np.array([cost[dcuts[r]:dcuts[r + 1]].sum() for r in range(4)]) / cost.sum()
    assert share.max() < dshare.max()
    assert share.max() < 0.5
    roots = np.sort(np.random.default_rng(3).choice(n, 500, replace=False)).astype(np.int32)
    pieces = [bench.shard_roots(roots, cost, 4, r) for r in range(4)]
    assert np.array_equal(np.concatenate(pieces), roots)
