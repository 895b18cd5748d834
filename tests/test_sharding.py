"""Multi-rank path of bench.py on CPU: world_size-2 gloo ranks each count
their start-node shard (the oracle stands in for a rank's GPU), and the
limb-wise all-reduce recovers the exact whole-graph counts."""
import os

import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

PATTERNS = {"ffl": synth.FFL, "cycle4": synth.CYCLE4, "bifan": synth.BIFAN}


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, src, dst = synth.er_graph(300, 2400, seed=21)
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


def test_two_rank_shards_sum_to_whole():
    import bench
    import oracle
    n, src, dst = synth.er_graph(300, 2400, seed=21)
    b = bench.shard_bounds(n, src, dst, 2)
    assert b[0][0] == 0 and b[-1][1] == n and b[0][1] == b[1][0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
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
