"""Oracle side of the R-MAT scale-24 parity test (test infrastructure).

tests/test_parity_s24.py starts this script as a process of its own, so that
it can fork worker processes that never held a CUDA context. It builds the
scale-24 workload graph (R-MAT scale 24, edge factor 16, a=.57 b=.19 c=.19,
seed 3) with the oracle, draws a seeded stratified start-node sample, and
writes the oracle's embedding counts per start node for each pattern (rooted
at the pattern vertex given in the spec), plus every embedding of a few start
nodes, to an .npz file. No value here comes from the GPU library.

Sample (per pattern):
  * uniform: `uniform` start nodes drawn without replacement (seeded); a
    node whose rooted walk would examine more than `cap_uniform` candidates
    is not counted (its count is marked unverified: the single-threaded walk
    is quadratic or worse in the degrees of hub neighbourhoods);
  * hubs: among the nodes whose estimated walk deg(v) x (sum of the total
    degrees of v's out- and in-neighbours) is at most `cap_hub`, those of
    highest total degree, in order, whose rooted walk finishes within
    `cap_hub` candidates, until `hubs` of them are counted (at most
    `hub_tries` attempts). The very top hubs need far more work than any cap
    a test can afford (a walk from node 0 examines ~10^13 candidates), so
    the hub stratum holds the heaviest nodes the oracle can still finish.

    python tests/s24_oracle_job.py spec.json out.npz
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import synth  # noqa: E402

_OG = None
_PATS = None


def _count(task):
    name, v, cap = task
    pat, root = _PATS[name]
    c = _OG.count_embeddings_capped(pat, root, v, v + 1, cap)
    return name, v, c


def main():
    global _OG, _PATS
    spec = json.load(open(sys.argv[1]))
    out_path = sys.argv[2]
    t0 = time.time()
    n, src, dst = synth.rmat24()
    _OG = oracle.OracleGraph(n, src, dst)
    del src, dst
    t_build = time.time() - t0
    off, adj = _OG.out_csr()
    outdeg = np.diff(off)
    deg = outdeg + np.bincount(adj, minlength=n)
    src_of = np.repeat(np.arange(n, dtype=np.int32), outdeg)
    nb_deg = np.bincount(src_of, weights=deg[adj], minlength=n) + np.bincount(adj, weights=deg[src_of], minlength=n)
    est = deg * nb_deg
    del off, adj, src_of, nb_deg
    _PATS = {name: ((p["k"], [tuple(a) for a in p["arcs"]]), p["root"]) for name, p in spec["patterns"].items()}
    rng = np.random.default_rng(spec["seed"])
    uniform = np.sort(rng.choice(n, spec["uniform"], replace=False)).astype(np.int64)
    light = np.nonzero(est <= spec["cap_hub"])[0]
    by_degree = light[np.argsort(-deg[light], kind="stable")]
    procs = spec.get("procs") or os.cpu_count() or 1
    results = {}
    with mp.get_context("fork").Pool(procs) as pool:
        # uniform stratum, all patterns at once
        tasks = [(name, int(v), spec["cap_uniform"]) for name in _PATS for v in uniform]
        for name, v, c in pool.imap_unordered(_count, tasks, chunksize=4):
            results[(name, v)] = c
        # hub stratum: candidates by descending degree, a batch at a time
        hubs = {name: [] for name in _PATS}
        tried = {name: 0 for name in _PATS}
        pos = 0
        while pos < spec["hub_tries"] and any(len(h) < spec["hubs"] for h in hubs.values()):
            batch = [int(v) for v in by_degree[pos: pos + procs]]
            pos += procs
            tasks = [(name, v, spec["cap_hub"]) for name in _PATS for v in batch if len(hubs[name]) < spec["hubs"]]
            for name, v, c in pool.map(_count, tasks, chunksize=1):
                tried[name] += 1
                if c is not None and len(hubs[name]) < spec["hubs"]:
                    hubs[name].append(v)
                    results[(name, v)] = c
    out = {"n": n, "build_s": t_build, "total_s": time.time() - t0, "procs": procs}
    for name in _PATS:
        roots = np.concatenate([uniform, np.array(hubs[name], np.int64)])
        counts = [results.get((name, int(v))) for v in roots]
        ok = np.array([c is not None for c in counts])
        vals = [c if c is not None else 0 for c in counts]
        out[f"{name}_roots"] = roots.astype(np.int32)
        out[f"{name}_hub"] = np.arange(len(roots)) >= len(uniform)
        out[f"{name}_ok"] = ok
        out[f"{name}_lo"] = np.array([c & 0xFFFFFFFFFFFFFFFF for c in vals], np.uint64)
        out[f"{name}_hi"] = np.array([c >> 64 for c in vals], np.uint64)
        out[f"{name}_hub_tries"] = tried[name]
        # every embedding of the first few verified uniform start nodes with matches
        pat, root = _PATS[name]
        ev = [int(v) for v, c in zip(uniform, counts[: len(uniform)])
              if c is not None and 0 < c <= spec["enum_max"]][: spec["enum_roots"]]
        rows = [_OG.enumerate_embeddings(pat, root, v, v + 1) for v in ev]
        out[f"{name}_enum_roots"] = np.array(ev, np.int32)
        out[f"{name}_enum_rows"] = np.concatenate(rows) if rows else np.zeros((0, pat[0]), np.int32)
    np.savez(out_path, **out)


if __name__ == "__main__":
    main()
