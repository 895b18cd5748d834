"""Benchmark: exact directed subgraph counting on one B300 (or N, sharded by start node).

Default workload: R-MAT scale 24 (2^24 nodes, edge factor 16, a=.57 b=.19
c=.19 d=.05, seed 3, deduplicated, self-loops dropped), dual CSR resident in
HBM; one step counts, over a seeded uniform sample of 1/4096 of the start
nodes, the matches of the directed 4-cycle, the bi-fan, the bi-parallel and
the 5-vertex feed-forward chain with one reciprocal arc (one xm_count_roots
call each; the chain through its cut-vertex split). Metric: matches/s =
matches found in the step / device time of the step. `--workload rmat20`
counts the 13 three-node motifs on R-MAT scale 20 instead.

    python bench.py [--gpus N --steps K --warmup W] [--workload rmat20|tiny|rmat22|rmat24|dense|batch|serve]
    python bench.py --impl reference ...      # the CPU oracle, bounded sample

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "matches/s"
# kernels one matching pass enqueues: first-level chunks, count, write (each
# followed by a 3-kernel scan except the write), units + scan, matcher
LAUNCHES_PER_CALL = 14
# bytes of one device plan copy (XmPlanDev: 8 levels and 7 product sets of
# 260 B, plus 52 B of header) and of the control block read back per pass
PLAN_BYTES = 52 + 15 * 260
CTL_BYTES = 24 * 8


def passes_per_call(plan, subset: bool):
    """Matching passes (and extra kernels) of one count call: a cut-vertex
    split runs one pass per part and per quotient plus a product kernel (over
    a start-node subset only when its plan description says so)."""
    sp = plan.split()
    if sp["cut"] < 0:
        return 1, 0
    if subset and "start-node subsets split" not in plan.describe():
        return 1, 0
    return len(sp["parts"]) + len(sp["quotients"]), 1
L2_FLUSH_BYTES = 512 << 20


def workload(name):
    if name == "tiny":
        n, src, dst = synth.tiny_er()
        pats = dict(synth.TINY_PATTERNS)
        desc = "directed ER n=2000 m=20000 seed 1; directed 3-cycle, feed-forward triangle, bi-fan"
    elif name == "rmat24":
        n, src, dst = synth.rmat24()
        pats = dict(synth.S24_PATTERNS)
        desc = "R-MAT scale 24 EF16 a=.57 b=.19 c=.19 seed 3; 4-cycle, bi-fan, bi-parallel, 5-vertex FF chain"
    elif name == "dense":
        n, src, dst = synth.rmat_graph(16, 8, seed=4)
        pats = {k: synth.DENSE_PATTERNS[k] for k in ("tt5", "tt6", "fan24")}
        desc = ("R-MAT scale 16 EF8 a=.57 b=.19 c=.19 seed 4; dense 5-6-vertex patterns: transitive "
                "tournaments on 5 and 6 vertices, 2x4 bipartite fan")
    elif name == "rmat22":
        n, src, dst = synth.rmat_graph(22, 16, seed=6)
        pats = dict(synth.S24_PATTERNS)
        desc = "R-MAT scale 22 EF16 a=.57 b=.19 c=.19 seed 6; 4-cycle, bi-fan, bi-parallel, 5-vertex FF chain"
    else:
        n, src, dst = synth.rmat20()
        pats = dict(synth.MOTIFS3)
        desc = "R-MAT scale 20 EF16 a=.57 b=.19 c=.19 seed 2; all 13 connected 3-node directed motifs, counts only"
    return n, src, dst, pats, desc


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_sha():
    h = hashlib.sha256()
    for f in ("xm_kernels.cu", "xm_kernels.cuh", "xm_plan_ir.h"):
        with open(os.path.join(ROOT, "paper_2404_11105_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name):
    """DRAM bytes per matcher launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        e = d[workload_name]
        if e.get("kernel_sha") == kernel_sha():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def start_node_sample(n, one_in):
    """The start nodes a sampled workload counts from: a seeded uniform
    sample of n // one_in nodes (the paper's runs from a percentage of the
    start nodes, Sec. 6.4), sorted."""
    rng = np.random.default_rng(24)
    roots = np.sort(rng.choice(n, n // one_in, replace=False)).astype(np.int32)
    return roots, f"start nodes: seeded uniform sample of 1/{one_in} ({len(roots)} nodes)"


# ------------------------------------------------------- sharding (N > 1) --

def root_costs(n, src, dst):
    """Estimated work of the walk from each start node: deg(v) times the
    summed degrees of v's neighbours (a walk extends v by each neighbour and
    each of those by its own list), plus one; total (out + in) degrees of the
    input arcs. On power-law graphs this grows much faster than deg(v)."""
    deg = np.bincount(src, minlength=n).astype(np.float64) + np.bincount(dst, minlength=n)
    nb = np.bincount(src, weights=deg[dst], minlength=n) + np.bincount(dst, weights=deg[src], minlength=n)
    return deg * nb + deg + 1.0


def balanced_cuts(cost, world):
    """Cut points 0 = c_0 <= ... <= c_world = len(cost) of contiguous pieces
    of about equal total cost."""
    cum = np.cumsum(cost)
    cuts = [0] + [int(np.searchsorted(cum, cum[-1] * r / world)) for r in range(1, world)] + [len(cost)]
    for r in range(1, len(cuts)):
        cuts[r] = min(max(cuts[r], cuts[r - 1]), len(cost))
    return cuts


def shard_bounds(n, src, dst, world):
    """Contiguous start-node ranges, one per rank, balanced by the estimated
    walk cost of their start nodes (root_costs); together they cover [0, n)
    exactly once."""
    if world <= 1:
        return [(0, n)]
    cuts = balanced_cuts(root_costs(n, src, dst), world)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_roots(roots, cost, world, rank):
    """Rank `rank`'s contiguous piece of the sorted start-node sample,
    balanced by the estimated cost of its start nodes."""
    if world <= 1:
        return roots
    cuts = balanced_cuts(cost[roots], world)
    return roots[cuts[rank]: cuts[rank + 1]]


def allreduce_counts(counts, dist, device="cpu"):
    """Sum exact (up to 2^93) per-pattern counts over ranks: each count is
    split into three 31-bit limbs so int64 sums cannot overflow."""
    t = __import__("torch").tensor([[c >> 62, (c >> 31) & 0x7FFFFFFF, c & 0x7FFFFFFF] for c in counts.values()],
                                   dtype=__import__("torch").int64, device=device)
    dist.all_reduce(t)
    return {name: (a << 62) + (b << 31) + c for name, (a, b, c) in zip(counts, t.cpu().tolist())}


# ----------------------------------------------------------- oracle (CPU) --

# a rooted oracle walk stops after this many candidates (some scale-24 start
# nodes would take it hours); its time still counts
ORACLE_ROOT_CAP = 20_000_000
_OG_CACHE = {}


def oracle_sample(n, src, dst, pats, budget_s, seed=0, roots=None):
    """The CPU oracle as it stands, single-threaded, on start nodes in seeded
    order (all nodes, or the given sample): embeddings rooted at pattern
    vertex 0, converted to matches (divided by |Aut|). Runs start nodes until
    budget_s per pattern. Returns (matches, seconds, start nodes, walks
    stopped at the cap)."""
    import oracle
    key = (n, len(src))
    if key not in _OG_CACHE:
        _OG_CACHE.clear()
        _OG_CACHE[key] = oracle.OracleGraph(n, src, dst)
    og = _OG_CACHE[key]
    rng = np.random.default_rng(seed)
    order = rng.permutation(n) if roots is None else rng.permutation(np.asarray(roots))
    per = budget_s / len(pats)
    matches = 0.0
    spent = 0.0
    nroots = 0
    gave_up = 0
    for pat in pats.values():
        aut = oracle.automorphisms(pat).shape[0]
        t0 = time.perf_counter()
        i = 0
        while time.perf_counter() - t0 < per and i < len(order):
            r = int(order[i])
            c = og.count_embeddings_capped(pat, 0, r, r + 1, ORACLE_ROOT_CAP)
            if c is None:
                gave_up += 1
            else:
                matches += c / aut
            i += 1
        spent += time.perf_counter() - t0
        nroots += i
    return matches, spent, nroots, gave_up


def _oracle_worker(job):
    """One process of the all-cores oracle baseline: builds the workload itself
    (untimed) and samples start nodes with its own seed for budget_s."""
    name, seed, budget_s, pattern_names = job
    n, src, dst, pats, _ = workload(name)
    if pattern_names:
        pats = {k: v for k, v in pats.items() if k in pattern_names}
    return oracle_sample(n, src, dst, pats, budget_s=budget_s, seed=1000 + seed)[:3]


def oracle_all_cores(name, pattern_names, procs, budget_s):
    """The oracle as it stands in `procs` concurrent processes (spawned), each
    on its own seeded start nodes: aggregate matches/s."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    jobs = [(name, i, budget_s, pattern_names) for i in range(procs)]
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, jobs))
    rate = sum(m / s for m, s, _ in res if s > 0)
    return rate, sum(r for _, _, r in res)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n, src, dst, pats, desc = workload(args.workload)
    if args.patterns:
        pats = {k: v for k, v in pats.items() if k in args.patterns.split(",")}
        desc += f" (subset: {','.join(pats)})"
    roots = None
    if args.workload in ("rmat22", "rmat24"):
        roots, sample_desc = start_node_sample(n, args.root_sample)
        desc += "; " + sample_desc
    vals = []
    last = None
    for step in range(args.warmup + args.steps):
        matches, secs, nroots, gave_up = oracle_sample(n, src, dst, pats, budget_s=args.ref_budget, seed=step,
                                                       roots=roots)
        if step >= args.warmup:
            vals.append(matches / secs)
            last = (nroots, secs, gave_up)
    v = statistics.median(vals)
    sample = ((f"{last[0]} start nodes of the same sample" if roots is not None else
               f"{last[0]} seeded uniform start nodes") +
              f" over the {len(pats)} patterns (~{args.ref_budget:.0f} s of single-threaded oracle time per step"
              + (f"; {last[2]} walks over {ORACLE_ROOT_CAP:.0e} candidates stopped, time counted, matches not"
                 if last[2] else "") + "); matches = rooted embeddings / |Aut|")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "matches/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * last[1], "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": v, "unit": "matches/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "matches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- serve arm ----

def run_serve(args):
    """Resident graphs, Poisson query arrivals, continuous batching into
    slots (one stream each) vs the same queries one xm_count at a time."""
    import torch
    import paper_2404_11105_b300 as xm

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    graphs = [xm.Graph(*synth.rmat_graph(22, 16, seed=6))]
    graphs += [xm.Graph(*synth.small_graph(i, seed=6, n_lo=100, n_hi=10000)) for i in range(args.serve_graphs)]
    load_s = time.perf_counter() - t0
    pool = [synth.batch_pattern(i, seed=66, k_hi=args.serve_kmax) for i in range(64)]
    plans = []
    for p in pool:
        pl = xm.Plan(p)
        pl.set_tuning(budget_ms=args.serve_budget_ms, blocks_per_sm=2)
        plans.append(pl)

    def requests(rate, seed):
        n = int(min(4000, max(200, rate * args.serve_seconds)))
        u = synth.uniforms(seed, 77, 3 * n).reshape(n, 3)
        arrivals = np.cumsum(-np.log1p(-u[:, 0]) / rate)
        pats = (u[:, 1] * len(plans)).astype(int)
        tgt = np.where(u[:, 2] < 0.1, 0, 1 + (u[:, 2] * 1e6).astype(int) % args.serve_graphs)
        return arrivals, pats, tgt

    def serve(rate, seed):
        arrivals, pats, tgt = requests(rate, seed)
        srv = xm.Server(graphs, slots=args.serve_slots, mem_budget_bytes=120 << 30)
        n = len(arrivals)
        done_t = np.zeros(n)
        status = np.zeros(n, int)
        counts = [None] * n
        nxt = 0
        start = time.perf_counter()
        finished = 0
        while finished < n:
            now = time.perf_counter() - start
            while nxt < n and arrivals[nxt] <= now:
                if not srv.submit(plans[pats[nxt]], int(tgt[nxt]), nxt):
                    break
                nxt += 1
            for tag, c, st in srv.poll(wait=False):
                done_t[tag] = time.perf_counter() - start
                status[tag] = st
                counts[tag] = c
                finished += 1
        srv.free()
        lat = (done_t - arrivals) * 1000.0
        ok = status == xm.XM_OK
        return {"rate_req_s": rate, "requests": n, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "completed_per_s": n / done_t.max(),
                "timeouts": int((status == xm.XM_ETIMEOUT).sum())}, counts, (arrivals, pats, tgt), ok

    results = []
    mixes = []
    for i, rate in enumerate(int(r) for r in args.serve_rates.split(",")):
        r, counts, req, ok = serve(rate, 100 + i)
        results.append(r)
        mixes.append((counts, req, ok))
    # the highest rate's requests one xm_count at a time (same budgets)
    counts, (arrivals, pats, tgt), ok = mixes[-1]
    t1 = time.perf_counter()
    same = 0
    n_seq = min(len(pats), 300)
    for q in range(n_seq):
        try:
            c = xm.xm_count(graphs[int(tgt[q])], plans[pats[q]])
        except xm.XmError as e:
            c = None
            assert e.status == xm.XM_ETIMEOUT
        if ok[q] and c is not None:
            assert c == counts[q], "a query's count differs alone and in the mix"
            same += 1
    seq_s = time.perf_counter() - t1
    seq_qps = n_seq / seq_s
    best = max(r["completed_per_s"] for r in results)
    line = {"metric": "queries/s", "value": best, "unit": "queries/s", "n_gpus": 1, "steps": len(results),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "resident R-MAT scale 22 EF16 (seed 6) + %d small graphs (n log-uniform "
                                   "100-10000, mean out-degree 4-12, seed 6); Poisson arrivals; random connected "
                                   "patterns k 3-%d, density 0.3-0.7; target scale-22 graph w.p. 0.1"
                                   % (args.serve_graphs, args.serve_kmax),
                       "slots": args.serve_slots, "budget_ms_per_query": args.serve_budget_ms,
                       "memory_budget_gb": 120, "graph_load_s": round(load_s, 1)},
            "per_rate": results,
            "sequential": {"queries_per_s": seq_qps, "queries": n_seq, "same_result_checked": same,
                           "sample": "first %d requests of the highest-rate stream, one xm_count each" % n_seq},
            "speedup_vs_sequential": best / seq_qps}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- batch arm ----

def run_batch(args):
    """Many patterns x many small graphs: one persistent launch (CUDA graph,
    autotuned) vs one launch per pattern vs one xm_count call per pair."""
    import torch
    import paper_2404_11105_b300 as xm

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    G, P = args.batch_graphs, args.batch_patterns
    t0 = time.perf_counter()
    graphs = [xm.Graph(*synth.small_graph(i, seed=5, n_hi=args.batch_nmax)) for i in range(G)]
    pats = [synth.batch_pattern(i, seed=4, k_hi=args.batch_kmax) for i in range(P)]
    plans = [xm.Plan(p) for p in pats]
    load_s = time.perf_counter() - t0
    pairs = [(pi, gi) for pi in range(P) for gi in range(G)]
    npairs = len(pairs)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return out

    budget = args.batch_pair_budget_ms
    batch = xm.Batch(plans, graphs, pairs)
    batch.set_pair_budget(budget)
    # autotuner on a sub-batch of pairs (every 16th pair), then applied to all
    sub = xm.Batch(plans, graphs, pairs[::16])
    sub.set_pair_budget(budget)
    cands = [(w, u, wpb, 0, 0, mr) for w in (128, 256) for u in (16, 64, 256) for wpb in (4, 8) for mr in (-1, 2)]
    best, best_ms = sub.tune(cands, reps=2)
    sub.free()
    batch.set_tuning(**best)
    for _ in range(args.warmup):
        batch.run(graph=True)
    torch.cuda.synchronize()
    counts = None

    def one_launch():
        nonlocal counts
        batch.run(graph=True)
        counts = batch.counts()

    with ClockSampler(0) as clk:
        ms_batch = timed(one_launch, args.steps)
    clocks = clk.summary()
    status = batch.pair_status()
    ok = status == xm.XM_OK
    # one launch per pattern (same kernel, P launches, same budgets)
    per_pattern = [xm.Batch([plans[pi]], graphs, [(0, gi) for gi in range(G)]) for pi in range(P)]
    for b in per_pattern:
        b.set_tuning(**best)
        b.set_pair_budget(budget)
    pp_counts, pp_ok = [], []

    def pattern_launches():
        pp_counts.clear()
        pp_ok.clear()
        for b in per_pattern:
            b.run()
        for b in per_pattern:
            pp_counts.extend(b.counts())
            pp_ok.extend((b.pair_status() == xm.XM_OK).tolist())

    ms_pp = timed(pattern_launches, max(1, args.steps // 2))
    both = [i for i in range(npairs) if ok[i] and pp_ok[i]]
    assert all(pp_counts[i] == counts[i] for i in both), "per-pattern launches disagree with the batched launch"
    # one xm_count call per pair on a seeded sample of the pairs that finished
    # within their budget, extrapolated to all pairs
    rng = np.random.default_rng(7)
    done = np.nonzero(ok)[0]
    sample = rng.choice(done, size=min(args.batch_single_sample, len(done)), replace=False)

    def singles():
        for i in sample:
            pi, gi = pairs[i]
            c = xm.xm_count(graphs[gi], plans[pi])
            assert c == counts[i]

    ms_single_sample = timed(singles, 1)[0]
    ms_single = ms_single_sample * npairs / len(sample)
    ms = statistics.median(ms_batch)
    total = sum(c for c, k in zip(counts, ok) if k)
    line = {"metric": "patterns/s", "value": npairs / (ms / 1000.0), "unit": "(pattern, graph) pairs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{P} random connected patterns (k 3-{args.batch_kmax}, density 0.3-0.7, seed 4) "
                                   f"x {G} small graphs (n log-uniform 50-{args.batch_nmax}, mean out-degree 4-12, "
                                   f"ER/R-MAT alternating, seed 5)", "pairs": npairs, "matches_per_step": total,
                       "pair_budget_ms": budget, "pairs_within_budget": int(ok.sum()),
                       "pairs_over_budget": int((~ok).sum()),
                       "graph_load_s": round(load_s, 1), "autotuned": best,
                       "autotune_sub_batch_ms": round(best_ms, 3)},
            "matches_per_s": total / (ms / 1000.0),
            "vs_one_launch_per_pattern": {"ms": statistics.median(ms_pp),
                                          "speedup": statistics.median(ms_pp) / ms},
            "vs_one_call_per_pair": {"ms_extrapolated": ms_single, "sample_pairs": int(len(sample)),
                                     "speedup": ms_single / ms,
                                     "how": "one xm_count per pair on a seeded sample of the pairs within budget, "
                                            "scaled to all pairs"},
            "gpu_launches": args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU arm ----

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xm", choices=["xm", "reference"])
    ap.add_argument("--workload", default="rmat24",
                    choices=["rmat20", "tiny", "rmat22", "rmat24", "dense", "batch", "serve"])
    ap.add_argument("--serve-graphs", type=int, default=1000)
    ap.add_argument("--serve-rates", default="100,300,1000,3000,10000")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window per rate")
    ap.add_argument("--serve-budget-ms", type=int, default=200, help="device-time budget per query")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-kmax", type=int, default=6)
    ap.add_argument("--batch-graphs", type=int, default=10000)
    ap.add_argument("--batch-patterns", type=int, default=256)
    ap.add_argument("--batch-kmax", type=int, default=6, help="largest pattern (vertices) in the batch")
    ap.add_argument("--batch-nmax", type=int, default=5000, help="largest graph (nodes) in the batch")
    ap.add_argument("--batch-single-sample", type=int, default=400,
                    help="pairs timed one xm_count call at a time (extrapolated)")
    ap.add_argument("--batch-pair-budget-ms", type=int, default=20,
                    help="device-time budget of each (pattern, graph) pair (0: none)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=4.0,
                    help="reference arm: seconds of single-threaded oracle time per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="also time the oracle in this many concurrent processes (-1: all host cores, at most 64)")
    ap.add_argument("--no-stats", action="store_true", help="skip the instrumented run (roofline bytes)")
    ap.add_argument("--patterns", default="", help="comma-separated subset of the workload's patterns")
    ap.add_argument("--root-sample", type=int, default=4096,
                    help="rmat22/rmat24: count over a seeded uniform sample of 1/N of the start nodes")
    ap.add_argument("--budget-ms", type=int, default=0, help="device-time budget per count call (0: none)")
    ap.add_argument("--merge-ratio", type=int, default=0,
                    help="intersection strategy threshold of two-list last levels (0: library default, -1: "
                         "never merge)")
    ap.add_argument("--no-tune", action="store_true", help="skip the per-pattern autotuner (warm-up phase)")
    ap.add_argument("--ablation", action="store_true",
                    help="also time every pattern with its unreduced plan (no candidate-set reuse)")
    ap.add_argument("--leaf-products", action="store_true",
                    help="also count leaf-product and cut-vertex-split patterns on the whole graph, each "
                         "against the level-by-level walk (budget --walk-budget-ms)")
    ap.add_argument("--walk-budget-ms", type=int, default=20000, help="0: skip the walks")
    ap.add_argument("--enum-capacity", type=int, default=1 << 24,
                    help="rmat24: matches written by the untimed enumeration check")
    ap.add_argument("--no-whole-ffchain", action="store_true",
                    help="rmat24: skip the whole-graph feed-forward chain count through the split")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)

    import torch
    import torch.distributed as dist
    import paper_2404_11105_b300 as xm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    n, src, dst, pats, desc = workload(args.workload)
    if args.patterns:
        keep = args.patterns.split(",")
        pats = {k: v for k, v in pats.items() if k in keep}
        desc += f" (subset: {','.join(pats)})"
    g = xm.Graph(n, src, dst)
    plans = {name: xm.Plan(p) for name, p in pats.items()}
    for p in plans.values():
        p.set_tuning(budget_ms=args.budget_ms, merge_ratio=args.merge_ratio)
    r_lo, r_hi = shard_bounds(n, src, dst, world)[rank]
    roots = None
    if args.workload in ("rmat22", "rmat24"):
        roots, sample_desc = start_node_sample(n, args.root_sample)
        if world > 1:
            roots = shard_roots(roots, root_costs(n, src, dst), world, rank)
        desc += "; " + sample_desc

    def count_one(p):
        if roots is not None:
            return xm.xm_count_roots(g, p, roots)
        return xm.xm_count_range(g, p, r_lo, r_hi) if world > 1 else xm.xm_count(g, p)

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        counts = {}
        for name, p in plans.items():
            counts[name] = count_one(p)
        if world > 1:
            counts = allreduce_counts(counts, dist, device="cuda")
        return counts

    tuned = {}
    if not args.no_tune and world == 1:
        # project autotuner (untimed, part of warm-up): window, unit size,
        # warps per block and the intersection strategy's length ratio, per
        # pattern on this graph (on the start-node sample when there is one)
        windows = (256,) if roots is not None else (256, 512)
        cands = [(w, u, wpb, 0, args.budget_ms, mr) for w in windows for wpb in (4, 8) for u in (8, 32)
                 for mr in ((args.merge_ratio,) if args.merge_ratio else (-1, 2))]
        for name, p in plans.items():
            best, _ = xm.xm_plan_tune(g, p, cands, reps=1, roots=roots)
            tuned[name] = {k: best[k] for k in ("window", "unit", "warps_per_block", "merge_ratio")}
    for _ in range(args.warmup):
        counts = step()

    kernel_ms = {name: [] for name in plans}
    prep_ms = {name: [] for name in plans}
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            counts = {}
            for name, p in plans.items():
                counts[name] = count_one(p)
                prep, match = g.last_timing()
                kernel_ms[name].append(match)
                prep_ms[name].append(prep)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    if world > 1:
        t = torch.tensor([max(step_ms)], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        counts = step()
        dist.barrier()
    clocks = clk.summary()
    ms = statistics.median(step_ms) if world == 1 else float(t.item())
    total_matches = sum(counts.values())
    value = total_matches / (ms / 1000.0)

    if rank != 0:
        dist.destroy_process_group()
        return 0

    # Roofline of the dominant kernel, the persistent matcher k_match (one
    # launch per pattern per step): its algorithmic bytes (an instrumented,
    # untimed run that takes the same code paths) over its own CUDA-event
    # time in the timed steps. The first-level pass before it (k_l1 and the
    # scans, prep_ms) gets its own line.
    peak, peak_kind = measured_peaks()
    per_pattern = {}
    alg_total = touched_total = l1_total = 0
    extensions = 0
    if not args.no_stats:
        for name, p in plans.items():
            if roots is not None:
                c, st = xm.xm_count_roots_stats(g, p, roots)
            else:
                c, st = xm.xm_count_stats(g, p, r_lo, r_hi)
            assert c == counts[name] or world > 1
            kms = statistics.median(kernel_ms[name])
            per_pattern[name] = {"matcher_ms": round(kms, 3), "prep_ms": round(statistics.median(prep_ms[name]), 3),
                                 "alg_bytes": st["alg_bytes"], "touched_bytes": st["touched_bytes"],
                                 "alg_gbs": round(st["alg_bytes"] / kms / 1e6, 1),
                                 "frac": round(st["alg_bytes"] / kms / 1e6 / peak, 4),
                                 "warp_exit_ms": [round(st[k] / 1e6, 2) for k in
                                                  ("warp_exit_first_ns", "warp_exit_mean_ns", "warp_exit_last_ns")]}
            alg_total += st["alg_bytes"]
            touched_total += st["touched_bytes"]
            l1_total += st["l1_bytes"]
            extensions += st["extensions"]
    kernel_s = sum(statistics.median(v) for v in kernel_ms.values()) / 1000.0   # per step
    prep_s = sum(statistics.median(v) for v in prep_ms.values()) / 1000.0
    launches = len(plans)
    achieved = alg_total / kernel_s / 1e9 if alg_total else None
    traffic = profiled_traffic(args.workload)   # ncu DRAM bytes per matcher launch, current kernel only
    # `achieved`/`frac`: algorithmic bytes per second of matcher time (the
    # bytes the plan's intersections need, each list scanned or probed,
    # whichever is cheaper, whether DRAM or L2 serves them); `dram_gbs` /
    # `dram_frac`: the DRAM traffic ncu measured on the same kernel source.
    # Algorithmic rates above the copy peak mean L2 serves the reuse: the
    # bound is then reported as "l2".
    roofline = {"bound": "hbm" if not achieved or achieved <= peak else "l2",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "basis": "algorithmic bytes (min(scan, probe) per list operand) / matcher device time",
                "traffic": traffic, "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_total / launches if alg_total else None,
                "kernel_ms_per_launch": kernel_s * 1000.0 / launches,
                "kernel": "k_match (persistent matcher)", "kernel_share_of_step": kernel_s * 1000.0 / ms,
                # DRAM bytes (ncu) per second of matcher time: the HBM traffic the kernel really moves
                "dram_gbs": None if traffic is None else traffic / (kernel_s / launches) / 1e9,
                "dram_frac": None if traffic is None else traffic / (kernel_s / launches) / 1e9 / peak,
                # bytes the chosen strategies would move with no cache, for comparison with DRAM traffic
                "touched_bytes_per_launch": touched_total / launches if touched_total else None,
                "frac_of_nominal": achieved / 7700.0 if achieved else None,
                "extensions_per_s": extensions / kernel_s if extensions else None,
                "per_pattern": per_pattern,
                "first_level_pass": {"alg_bytes": l1_total, "ms": round(prep_s * 1000.0, 3),
                                     "alg_gbs": round(l1_total / prep_s / 1e9, 1) if prep_s else None}}

    ablation = None
    if args.ablation:
        # reduced plan vs the plan over the original pattern (no reduction,
        # no reuse): device time, algorithmic bytes, equal counts
        ablation = {}
        for name, pat in pats.items():
            row = {}
            for label, flags in (("reduced", xm.XM_REDUCE), ("unreduced", xm.XM_NO_REDUCE)):
                p = xm.Plan(pat, flags)
                if args.budget_ms:
                    p.set_tuning(budget_ms=args.budget_ms)
                ms_ = []
                try:
                    for _ in range(3):
                        c = count_one(p)
                        ms_.append(sum(g.last_timing()))
                except xm.XmError as e:
                    if e.status != xm.XM_ETIMEOUT:
                        raise
                    row[label] = {"timed_out": True, "budget_ms": args.budget_ms, "reuse_levels": p.n_reuse}
                    continue
                assert c == counts[name]
                if roots is not None:
                    _, st = xm.xm_count_roots_stats(g, p, roots)
                else:
                    _, st = xm.xm_count_stats(g, p, r_lo, r_hi)
                row[label] = {"ms": round(min(ms_), 3), "alg_bytes": st["alg_bytes"], "reuse_levels": p.n_reuse}
            if "ms" in row["unreduced"] and "ms" in row["reduced"]:
                row["speedup"] = round(row["unreduced"]["ms"] / row["reduced"]["ms"], 3)
            ablation[name] = row

    products = None
    if args.leaf_products:
        # whole-graph counts that stop early (Sec. 5.3 products, cut-vertex
        # splits) against the plain walk of every level; wall time of the
        # xm_count call (a split runs several launches and host steps)
        products = {}
        pats_next = dict(synth.LEAF_PRODUCT_PATTERNS) if args.workload != "rmat24" else {}
        pats_next.update(synth.SPLIT_PATTERNS if args.workload != "rmat24" else {"ffchain5": synth.FFCHAIN5})
        for name, pat in pats_next.items():
            row = {}
            for label, flags in (("early", xm.XM_REDUCE), ("walk", xm.XM_NO_PRODUCT | xm.XM_NO_SPLIT)):
                if label == "walk" and (args.workload == "rmat24" or args.walk_budget_ms <= 0):
                    continue
                p = xm.Plan(pat, flags)
                p.set_tuning(budget_ms=max(args.walk_budget_ms, 0))
                best = None
                for _ in range(1 if label == "walk" else 3):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    try:
                        c = xm.xm_count(g, p)
                    except xm.XmError as e:
                        if e.status != xm.XM_ETIMEOUT:
                            raise
                        c = None
                    torch.cuda.synchronize()
                    t = (time.perf_counter() - t0) * 1e3
                    best = t if best is None else min(best, t)
                    if c is None:
                        break
                row[label] = {"count": None if c is None else int(c), "ms": round(best, 2),
                              "timed_out": c is None}
            pe = xm.Plan(pat)
            pr, sp = pe.product(), pe.split()
            row["product"] = {"level": pr["level"], "r": pr["r"], "kind": pr["kind"]} if pr["r"] else None
            row["split"] = {"cut": sp["cut"], "parts": len(sp["parts"]), "quotients": len(sp["quotients"])} \
                if sp["cut"] >= 0 else None
            if "walk" in row and row["walk"]["count"] is not None:
                assert row["walk"]["count"] == row["early"]["count"], name
                row["speedup"] = round(row["walk"]["ms"] / row["early"]["ms"], 2)
            products[name] = row

    enum = None
    if roots is not None and args.enum_capacity > 0:
        # enumeration into a device buffer (untimed): the first pattern
        name0, p0 = next(iter(plans.items()))
        out = torch.empty(args.enum_capacity * p0.k, dtype=torch.int32, device="cuda")
        total, written, over = xm.xm_enumerate_roots(g, p0, roots, out)
        assert total == counts[name0]
        rows = out[: written * p0.k].view(-1, p0.k)
        enum = {"pattern": name0, "total": int(total), "written": int(written), "overflow": bool(over),
                "capacity": args.enum_capacity,
                "start_nodes_in_sample": bool(torch.isin(rows[:, p0.start].cpu(),
                                                         torch.from_numpy(roots)).all().item()) if written else True}
        del out

    # end to end through the public API with host buffers: pinned arc arrays
    # -> xm_load_graph (upload, dual CSR and hash index built on the device)
    # -> the step's counts -> readback
    e2e = None
    if args.e2e_steps > 0:
        hs = torch.from_numpy(src).pin_memory()
        hd = torch.from_numpy(dst).pin_memory()
        e2e_ms = []
        h2d = 0
        for _ in range(args.e2e_steps):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            g2 = xm.Graph(n, hs, hd)
            c2 = {name: (xm.xm_count_roots(g2, p, roots) if roots is not None else xm.xm_count(g2, p))
                  for name, p in plans.items()}
            ev1.record(stream)
            ev1.synchronize()
            e2e_ms.append(ev0.elapsed_time(ev1))
            g2.free()
            assert c2 == counts
        # host -> device: the arc arrays, then per matching pass one plan copy
        # and (sampled workloads) the staged start-node list; device -> host:
        # per pass the control block (counts, status), per split its product
        npass = sum(passes_per_call(p, roots is not None)[0] for p in plans.values())
        nsplit = sum(passes_per_call(p, roots is not None)[1] for p in plans.values())
        h2d = hs.numel() * 4 + hd.numel() * 4 + npass * PLAN_BYTES + \
            (len(plans) * roots.size * 4 if roots is not None else 0)
        d2h = npass * CTL_BYTES + nsplit * 16
        e2e = {"value": total_matches / (statistics.median(e2e_ms) / 1000.0), "unit": "matches/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": statistics.median(e2e_ms)}

    # the whole-graph count of the 5-vertex feed-forward chain through its
    # cut-vertex decomposition (part counts per node, product sum, quotient
    # counts: several launches and host steps), beside the sampled step
    whole = None
    if args.workload == "rmat24" and "ffchain5" in pats and not args.no_whole_ffchain:
        pw = xm.Plan(synth.FFCHAIN5)
        wms = []
        for _ in range(3):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            cw = xm.xm_count(g, pw)
            ev1.record(stream)
            ev1.synchronize()
            wms.append(ev0.elapsed_time(ev1))
        sp = pw.split()
        whole = {"pattern": "ffchain5", "count": int(cw), "ms": round(min(wms), 2),
                 "matches_per_s": cw / (min(wms) / 1000.0),
                 "how": f"cut vertex {sp['cut']}: {len(sp['parts'])} rooted part counts per node, "
                        f"{len(sp['quotients'])} quotient patterns (not in the timed step)"}

    cpu = None
    if not args.no_cpu_baseline:
        m_, s_, nr, gave_up = oracle_sample(n, src, dst, pats, budget_s=args.cpu_budget, roots=roots)
        cpu = {"value": m_ / s_, "unit": "matches/s", "cores": 1, "kind": "oracle",
               "sample": (f"{nr} start nodes of the same sample" if roots is not None else
                          f"{nr} seeded uniform start nodes") +
                         f" over the {len(pats)} patterns, {s_:.1f} s single-threaded"
                         + (f" ({gave_up} walks over {ORACLE_ROOT_CAP:.0e} candidates stopped, their time "
                            f"counted, their matches not)" if gave_up else "")
                         + "; matches = rooted embeddings / |Aut|"}
        if args.cpu_procs:
            procs = min(os.cpu_count() or 1, 64) if args.cpu_procs < 0 else args.cpu_procs
            rate, nr_all = oracle_all_cores(args.workload, list(pats), procs, args.cpu_budget)
            cpu["all_cores"] = {"value": rate, "unit": "matches/s", "cores": procs,
                                "sample": f"{nr_all} seeded start nodes in {procs} concurrent processes, "
                                          f"~{args.cpu_budget:.0f} s each"}

    line = {"metric": METRIC, "value": value, "unit": "matches/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "ms_per_step_min_max": [min(step_ms), max(step_ms)],
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "graph_nodes": g.n, "graph_arcs": g.m, "patterns": len(plans),
                       "matches_per_step": total_matches, "l2": "flushed (512 MB write) between timed steps",
                       "parallelism": f"start-node shards x{world}" if world > 1 else "1 GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": sum(LAUNCHES_PER_CALL * a + b for a, b in
                                (passes_per_call(p, roots is not None or world > 1) for p in plans.values()))
                            * args.steps, "clocks": clocks,
            "counts": {k: int(v) for k, v in counts.items()}, "whole_graph": whole, "enumeration": enum,
            "ablation": ablation, "leaf_products": products,
            "autotuned": tuned,
            "device_ms_per_pattern": {k: round(statistics.median(kernel_ms[k]) + statistics.median(prep_ms[k]), 3)
                                      for k in plans}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
