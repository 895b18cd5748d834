"""Writes rmat20_triangles.json: the feed-forward triangle count sum(A o A^2)
and the directed 3-cycle count tr(A^3)/3 of the R-MAT scale-20 workload
graph (edge factor 16, a=.57 b=.19 c=.19, seed 2, repeats and self-loops
dropped), computed by the CPU oracle alone (og_triangle_sums: one sorted-list
intersection per arc), in worker processes over interleaved source ranges.

    python tests/golden/make_rmat20_triangles.py [--procs N]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

_G = None


def _init():
    global _G
    n, src, dst = synth.rmat20()
    _G = oracle.OracleGraph(n, src, dst)


def _part(rng):
    return _G.triangle_sums(*rng)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    n = 1 << 20
    step = 1024
    ranges = [(a, min(n, a + step)) for a in range(0, n, step)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.procs, initializer=_init) as pool:
        parts = pool.map(_part, ranges, chunksize=1)
    ffl = sum(p[0] for p in parts)
    walks = sum(p[1] for p in parts)
    assert walks % 3 == 0
    out = {"graph": "R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19 d=.05, seed 2, repeats and self-loops "
                    "dropped (synth.rmat20)",
           "method": "oracle og_triangle_sums over all arcs",
           "030T_feed_forward_triangles": ffl, "030C_directed_3_cycles": walks // 3}
    with open(os.path.join(HERE, "rmat20_triangles.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out, f"{time.time() - t0:.0f} s on {args.procs} processes")


if __name__ == "__main__":
    main()
