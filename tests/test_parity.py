"""GPU parity: the CUDA matcher (through the C ABI) against the CPU oracle.

Counts must be bit-exact; enumerated match sets must be equal after the
oracle's canonicalisation (each match written once, in any order).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def xm():
    import paper_2404_11105_b300 as m
    return m


def graph_pair(xm, n, src, dst):
    return xm.Graph(n, src, dst), oracle.OracleGraph(n, src, dst)


# launch shapes, and the three intersection strategies of two-list last
# levels: the default length-ratio choice, merging whenever possible
# (merge_ratio 1024) and never merging (probes only)
TUNINGS = [dict(), dict(window=64, unit=1, warps_per_block=2, merge_ratio=1024),
           dict(window=96, unit=7, warps_per_block=4, merge_ratio=-1),
           dict(window=128, unit=3, warps_per_block=1, blocks_per_sm=1, merge_ratio=1)]

NAMED = {"cycle3": synth.CYCLE3, "ffl": synth.FFL, "bifan": synth.BIFAN, "cycle4": synth.CYCLE4,
         "biparallel": synth.BIPARALLEL, "ffchain5": synth.FFCHAIN5}


def random_patterns(count, seed):
    pats = []
    for i in range(count):
        u = synth.uniforms(seed, 1000 + i, 2)
        pats.append(synth.random_pattern(3 + int(u[0] * 4), 0.3 + 0.4 * u[1], seed, i))
    return pats


# ------------------------------------------------------- tiny ER (config 0)

@pytest.fixture(scope="module")
def tiny(xm):
    n, src, dst = synth.tiny_er()
    return graph_pair(xm, n, src, dst)


@pytest.mark.parametrize("name", ["cycle3", "ffl", "bifan"])
def test_tiny_counts_and_sets(xm, tiny, name):
    g, og = tiny
    pat = NAMED[name]
    want = og.count_matches(pat)
    ref_rows = og.enumerate(pat)
    assert ref_rows.shape[0] == want
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE):
        for tun in TUNINGS:
            p = xm.Plan(pat, flags)
            p.set_tuning(**tun)
            assert xm.xm_count(g, p) == want, (flags, tun)
            out = torch.full((max(want, 1) * pat[0],), -1, dtype=torch.int32, device="cuda")
            total, written, over = xm.xm_enumerate(g, p, out)
            assert (total, written, over) == (want, want, False)
            rows = out[: want * pat[0]].view(-1, pat[0]).cpu().numpy()
            canon = oracle.canonicalize(pat, rows)
            assert np.array_equal(canon, ref_rows)
            # each match written once
            assert np.unique(canon, axis=0).shape[0] == want
    pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
    assert xm.xm_count(g, pe) == og.count_embeddings(pat)


@pytest.mark.parametrize("name", sorted(synth.MOTIFS3))
def test_tiny_motifs(xm, tiny, name):
    g, og = tiny
    pat = synth.MOTIFS3[name]
    want = og.count_matches(pat)
    for tun in TUNINGS[:2]:
        p = xm.Plan(pat)
        p.set_tuning(**tun)
        assert xm.xm_count(g, p) == want


def test_tiny_enumerate_overflow(xm, tiny):
    g, og = tiny
    pat = synth.BIFAN
    want = og.count_matches(pat)
    cap = max(1, want // 3)
    p = xm.Plan(pat)
    out = torch.full((cap * 4,), -1, dtype=torch.int32, device="cuda")
    total, written, over = xm.xm_enumerate(g, p, out, capacity=cap)
    assert over and total == want and written == cap
    rows = oracle.canonicalize(pat, out.view(-1, 4).cpu().numpy())
    ref = {tuple(r) for r in og.enumerate(pat).tolist()}
    assert all(tuple(r) in ref for r in rows.tolist())
    assert np.unique(rows, axis=0).shape[0] == cap


# ------------------------------------------ small skewed graphs, many tiles

@pytest.fixture(scope="module")
def rmat_small(xm):
    # R-MAT scale 10, edge factor 6: skewed (hubs of a few hundred arcs),
    # small enough for the single-threaded oracle to finish in seconds
    n, src, dst = synth.rmat_graph(10, 6, seed=17)
    return graph_pair(xm, n, src, dst)


@pytest.fixture(scope="module")
def rmat_tiny(xm):
    # R-MAT scale 9, edge factor 8, for random patterns of up to 6 vertices
    n, src, dst = synth.rmat_graph(9, 8, seed=17)
    return graph_pair(xm, n, src, dst)


@pytest.mark.parametrize("name", list(NAMED))
def test_rmat_small_named(xm, rmat_small, name):
    g, og = rmat_small
    pat = NAMED[name]
    want = og.count_matches(pat)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE):
        for tun in TUNINGS:
            p = xm.Plan(pat, flags)
            p.set_tuning(**tun)
            assert xm.xm_count(g, p) == want, (flags, tun)
    pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
    assert xm.xm_count(g, pe) == og.count_embeddings(pat)


@pytest.mark.parametrize("pattern", random_patterns(16, 5))
def test_rmat_small_random_patterns(xm, rmat_tiny, pattern):
    g, og = rmat_tiny
    want = og.count_matches(pattern)
    for tun in (TUNINGS[0], TUNINGS[1]):
        p = xm.Plan(pattern)
        p.set_tuning(**tun)
        assert xm.xm_count(g, p) == want


def test_root_range_additivity(xm, rmat_small):
    g, og = rmat_small
    for pat in (synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5):
        p = xm.Plan(pat)
        whole = xm.xm_count(g, p)
        cuts = [0, 1, 2, 17, 300, 1024, g.n]
        parts = sum(xm.xm_count_range(g, p, a, b) for a, b in zip(cuts, cuts[1:]))
        assert parts == whole
        # per start node, in embeddings mode: the oracle rooted at the plan's start vertex
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
        for r in (0, 1, 5, 77, 1000):
            assert xm.xm_count_range(g, pe, r, r + 1) == og.count_embeddings(pat, pe.start, r, r + 1)


def test_count_roots_each(xm, rmat_small):
    """Per-start-node counts in one launch: each equals the oracle rooted at
    the plan's start vertex (embeddings mode) and the one-node range count
    (matches); repeated and unsorted nodes keep the caller's order; the
    per-node counts add up to xm_count_roots; leaf-product plans too."""
    g, og = rmat_small
    rng = np.random.default_rng(8)
    roots = np.concatenate([rng.integers(0, g.n, 40), [0, 1, 2, 0, 7, g.n - 1]]).astype(np.int32)
    for pat in (synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL, synth.FFCHAIN5, synth.FFL,
                PRODUCT_PATTERNS["path4"], (2, [(0, 1)])):
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS | xm.XM_NO_SPLIT)
        for tun in (TUNINGS[0], TUNINGS[1], TUNINGS[2]):
            pe.set_tuning(**tun)
            got = xm.xm_count_roots_each(g, pe, roots)
            want = [og.count_embeddings(pat, pe.start, v, v + 1) for v in roots.tolist()]
            assert got == want, (pat, tun)
        p = xm.Plan(pat)
        per = xm.xm_count_roots_each(g, p, roots)
        assert per == [xm.xm_count_range(g, p, v, v + 1) for v in roots.tolist()]
        uniq = np.unique(roots)
        assert sum(xm.xm_count_roots_each(g, p, uniq)) == xm.xm_count_roots(g, p, uniq)
    assert xm.xm_count_roots_each(g, xm.Plan(synth.BIFAN), np.zeros(0, np.int32)) == []
    with pytest.raises(xm.XmError):
        xm.xm_count_roots_each(g, xm.Plan(synth.BIFAN), np.array([-1], np.int32))


def test_enumerate_sets_rmat_small(xm, rmat_small):
    g, og = rmat_small
    for pat in (synth.FFL, synth.CYCLE4, synth.FFCHAIN5):
        want = og.count_matches(pat)
        ref = og.enumerate(pat)
        p = xm.Plan(pat)
        p.set_tuning(window=64, unit=5)
        out = torch.full((max(want, 1) * pat[0],), -1, dtype=torch.int32, device="cuda")
        total, written, over = xm.xm_enumerate(g, p, out)
        assert total == want and written == want and not over
        rows = oracle.canonicalize(pat, out[: want * pat[0]].view(-1, pat[0]).cpu().numpy())
        assert np.array_equal(rows, ref)


# ------------------------------------------------------------- edge cases

def test_edge_cases(xm):
    # no arcs at all
    g = xm.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.m == 0
    assert xm.xm_count(g, xm.Plan(synth.CYCLE3)) == 0
    # self-loops and repeats only
    g = xm.Graph(3, np.array([0, 1, 1, 2, 2], np.int32), np.array([0, 1, 2, 1, 1], np.int32))
    assert g.m == 2
    assert xm.xm_count(g, xm.Plan((2, [(0, 1)]))) == 2
    assert xm.xm_count(g, xm.Plan((2, [(0, 1), (1, 0)]))) == 1
    # single arc pattern counts arcs; reciprocal pair counts reciprocal pairs
    n, src, dst = synth.er_graph(500, 6000, seed=9)
    g, og = graph_pair(xm, n, src, dst)
    assert xm.xm_count(g, xm.Plan((2, [(0, 1)]))) == og.m
    assert xm.xm_count(g, xm.Plan((2, [(0, 1), (1, 0)]))) == og.count_matches((2, [(0, 1), (1, 0)]))
    # empty root range, out-of-range root range
    p = xm.Plan(synth.FFL)
    assert xm.xm_count_range(g, p, 10, 10) == 0
    assert xm.xm_count_range(g, p, n + 5, n + 50) == 0
    assert xm.xm_count_range(g, p, -100, n + 100) == xm.xm_count(g, p)
    # enumerate with capacity 0: exact total, overflow flagged
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    total, written, over = xm.xm_enumerate(g, p, out, capacity=0)
    assert total == og.count_matches(synth.FFL) and written == 0 and over == (total > 0)
    # complete digraph (dense lists, every candidate survives)
    k7 = [(u, v) for u in range(24) for v in range(24) if u != v]
    g, og = graph_pair(xm, 24, np.array([a for a, _ in k7], np.int32), np.array([b for _, b in k7], np.int32))
    for pat in (synth.CYCLE4, synth.BIFAN, synth.FFCHAIN5):
        assert xm.xm_count(g, xm.Plan(pat)) == og.count_matches(pat)


def _oracle_dual_csr(og):
    """The oracle's sorted adjacency as out- and in-CSR (the in-lists as
    the transpose of its out-lists)."""
    off, adj = og.out_csr()
    src = np.repeat(np.arange(og.n, dtype=np.int64), np.diff(off))
    order = np.lexsort((src, adj))
    in_adj = src[order].astype(np.int32)
    in_off = np.concatenate([[0], np.cumsum(np.bincount(adj, minlength=og.n))]).astype(np.int64)
    return off, adj, in_off, in_adj


def test_device_csr_build_against_oracle(xm):
    """The dual CSR built on the device (radix sort of packed arcs, repeats and
    self-loops dropped) equals the oracle's adjacency: skewed and uniform
    graphs with repeats and self-loops, a node without arcs, only loops,
    no arcs, device-pointer input, several builds in a row."""
    rng = np.random.default_rng(11)
    cases = [synth.rmat_graph(12, 8, seed=3), synth.er_graph(3000, 40000, seed=5)]
    n, s_, d_ = synth.rmat_graph(10, 16, seed=9)
    cases.append((n, np.concatenate([s_, s_[:5000], np.arange(50, dtype=np.int32)]),
                  np.concatenate([d_, d_[:5000], np.arange(50, dtype=np.int32)])))  # repeats and loops
    cases.append((7, np.array([0, 1, 2, 2, 5], np.int32), np.array([1, 0, 2, 5, 2], np.int32)))  # node 6 isolated
    cases.append((4, np.array([1, 1, 3], np.int32), np.array([1, 1, 3], np.int32)))             # only loops
    cases.append((9, np.zeros(0, np.int32), np.zeros(0, np.int32)))                               # no arcs
    cases.append((1 << 15, rng.integers(0, 1 << 15, 200000).astype(np.int32),
                  rng.integers(0, 1 << 15, 200000).astype(np.int32)))
    for i, (n, src, dst) in enumerate(cases + cases[:2]):
        og = oracle.OracleGraph(n, src, dst)
        want = _oracle_dual_csr(og)
        for dev in ((False, True) if i == 0 else (False,)):
            a, b = (torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()) if dev else (src, dst)
            g = xm.Graph(n, a, b)
            assert g.m == og.m, i
            for got, w, name in zip(g.csr_host(), want, ("out_off", "out_adj", "in_off", "in_adj")):
                assert np.array_equal(got.astype(np.int64), np.asarray(w, np.int64)), (i, name)
            g.free()
    # an endpoint outside [0, n) is refused, for host and device arrays
    for dev in (False, True):
        s_bad = np.array([0, 1, 5], np.int32)
        d_bad = np.array([1, 2, 0], np.int32)
        a, b = (torch.from_numpy(s_bad).cuda(), torch.from_numpy(d_bad).cuda()) if dev else (s_bad, d_bad)
        with pytest.raises(xm.XmError) as ei:
            xm.Graph(4, a, b)
        assert ei.value.status == xm.XM_EINVAL


def test_device_pointer_input(xm):
    n, src, dst = synth.er_graph(800, 9000, seed=12)
    g1 = xm.Graph(n, src, dst)
    g2 = xm.Graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    assert g1.m == g2.m
    p = xm.Plan(synth.BIFAN)
    assert xm.xm_count(g1, p) == xm.xm_count(g2, p)


def test_stats_counters(xm, rmat_small):
    g, og = rmat_small
    p = xm.Plan(synth.BIFAN)
    c, st = xm.xm_count_stats(g, p)
    assert c == og.count_matches(synth.BIFAN)
    assert st["alg_bytes"] > 0 and st["units"] > 0 and st["extensions"] > 0
    prep, match = g.last_timing()
    assert prep >= 0 and match > 0


# ------------------------------------- full-size R-MAT scale 20 (config 1)

@pytest.fixture(scope="module")
def s20(xm):
    n, src, dst = synth.rmat20()
    g = xm.Graph(n, src, dst)
    og = oracle.OracleGraph(n, src, dst)
    return g, og


def test_s20_triangles_closed_forms(xm, s20):
    """The two triangle motifs on the whole scale-20 graph against the
    oracle's closed forms (tests/golden/rmat20_triangles.json, written by
    make_rmat20_triangles.py from the oracle alone): feed-forward triangles
    sum(A o A^2) and directed 3-cycles tr(A^3)/3, under every intersection
    strategy (length-ratio choice, always merge, never merge)."""
    import json
    import os
    g, og = s20
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rmat20_triangles.json")))
    for name, key in (("030T", "030T_feed_forward_triangles"), ("030C", "030C_directed_3_cycles")):
        for ratio in (0, 1024, -1):
            p = xm.Plan(synth.MOTIFS3[name])
            p.set_tuning(merge_ratio=ratio)
            assert xm.xm_count(g, p) == gold[key], (name, ratio)


def s20_roots(og, hubs=12, uniform=48, seed=20):
    """Start nodes for per-node checks on the scale-20 graph: the nodes of
    highest degree whose rooted walks the oracle still finishes in about a
    second (total degree at most 6000: the top hubs, of degree up to ~50,000,
    would take the single-threaded oracle minutes per motif) and seeded
    uniform nodes."""
    off, adj = og.out_csr()
    outdeg = np.diff(off)
    indeg = np.bincount(adj, minlength=og.n)
    deg = outdeg + indeg
    heavy = np.nonzero(deg <= 6000)[0]
    heavy = heavy[np.argsort(-deg[heavy], kind="stable")][:hubs]
    rng = np.random.default_rng(seed)
    return np.concatenate([heavy, rng.integers(0, og.n, uniform)]).astype(np.int32), deg


def test_s20_motifs_per_root_with_hubs(xm, s20):
    """All 13 motifs at full size: per-start-node embedding counts (one launch
    per motif through xm_count_roots_each) against the oracle rooted at the
    plan's start vertex, on hub nodes of degree 1500-6000 -- whose work is
    split into many 1024-id pieces -- and uniform nodes."""
    g, og = s20
    roots, deg = s20_roots(og)
    assert (deg[roots[:12]] > 1500).all()
    for name, pat in synth.MOTIFS3.items():
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
        got = xm.xm_count_roots_each(g, pe, roots)
        for v, c in zip(roots.tolist(), got):
            assert c == og.count_embeddings(pat, pe.start, v, v + 1), (name, v)


def test_s20_motifs_sampled_and_closed_forms(xm, s20):
    """All 13 motifs at full size in the bench's launch configuration:
    closed forms where they are cheap (stars, 2-path), reduced == unreduced
    on the whole graph, one-node ranges == per-node counts (hub nodes 0-3
    included)."""
    g, og = s20
    off, adj = og.out_csr()
    outdeg = np.diff(off)
    indeg = np.bincount(adj, minlength=og.n)
    # reciprocal partners per node
    src_of = np.repeat(np.arange(og.n, dtype=np.int64), outdeg)
    key = src_of * og.n + adj                      # ascending: CSR order
    rkey = adj.astype(np.int64) * og.n + src_of
    pos = np.minimum(np.searchsorted(key, rkey), key.size - 1)
    r = np.bincount(src_of[key[pos] == rkey], minlength=og.n)
    c2 = lambda x: (x * (x - 1) // 2).sum()
    assert xm.xm_count(g, xm.Plan(synth.MOTIFS3["021D"])) == int(c2(outdeg.astype(object)))
    assert xm.xm_count(g, xm.Plan(synth.MOTIFS3["021U"])) == int(c2(indeg.astype(object)))
    assert xm.xm_count(g, xm.Plan(synth.MOTIFS3["021C"])) == int((indeg.astype(object) * outdeg - r).sum())
    for name, pat in synth.MOTIFS3.items():
        red = xm.xm_count(g, xm.Plan(pat))
        assert red == xm.xm_count(g, xm.Plan(pat, xm.XM_NO_REDUCE)), name
        # per start node, through the one-node range entry point
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
        for v in (0, 1, 2, 3, 12345, og.n - 1):
            assert xm.xm_count_range(g, pe, v, v + 1) == xm.xm_count_roots_each(g, pe, [v])[0], (name, v)


DENSE = [synth.random_pattern(k, 0.9, 123, k) for k in (6, 7, 8)] + \
        [synth.random_pattern(6, 0.6, 7, s) for s in range(3)]


@pytest.mark.parametrize("pattern", DENSE)
def test_dense_patterns_many_operands(xm, rmat_tiny, pattern):
    # levels with more than 7 operand lists (reciprocal arcs to many earlier levels)
    g, og = rmat_tiny
    want = og.count_matches(pattern)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE):
        assert xm.xm_count(g, xm.Plan(pattern, flags)) == want
    assert xm.xm_count_batch([xm.Plan(pattern)], [g], [(0, 0)]) == [want]


def test_root_lists(xm, rmat_small):
    """Counts over explicit start-node lists: a random partition adds up to
    the whole count; per start node in embeddings mode they equal the
    oracle rooted at the plan's start vertex; enumeration over a root list
    gives exactly the matches of those start nodes."""
    g, og = rmat_small
    rng = np.random.default_rng(3)
    perm = rng.permutation(g.n).astype(np.int32)
    parts = np.array_split(perm, 5)
    for pat in (synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5, (2, [(0, 1)])):
        p = xm.Plan(pat)
        assert sum(xm.xm_count_roots(g, p, part) for part in parts) == xm.xm_count(g, p)
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
        sample = perm[:20]
        assert xm.xm_count_roots(g, pe, sample) == sum(og.count_embeddings(pat, pe.start, int(v), int(v) + 1)
                                                       for v in sample)
    # duplicates are ignored; empty list counts nothing
    p = xm.Plan(synth.CYCLE4)
    assert xm.xm_count_roots(g, p, np.concatenate([parts[0], parts[0]])) == xm.xm_count_roots(g, p, parts[0])
    assert xm.xm_count_roots(g, p, np.zeros(0, np.int32)) == 0
    with pytest.raises(xm.XmError):
        xm.xm_count_roots(g, p, np.array([g.n], np.int32))
    want = xm.xm_count_roots(g, p, parts[1])
    out = torch.full((max(want, 1) * 4,), -1, dtype=torch.int32, device="cuda")
    total, written, over = xm.xm_enumerate_roots(g, p, parts[1], out)
    assert total == want == written and not over
    rows = out[: want * 4].view(-1, 4).cpu().numpy()
    start_col = rows[:, p.start]
    assert np.isin(start_col, parts[1]).all()


@pytest.mark.parametrize("name", ["cycle3", "ffl", "bifan", "cycle4", "biparallel", "ffchain5"])
def test_induced_counts(xm, rmat_small, tiny, name):
    pat = NAMED[name]
    for g, og in (rmat_small, tiny):
        want = og.count_matches(pat, induced=True)
        for flags in (xm.XM_INDUCED, xm.XM_INDUCED | xm.XM_NO_REDUCE):
            for tun in TUNINGS[:2]:
                p = xm.Plan(pat, flags)
                p.set_tuning(**tun)
                assert xm.xm_count(g, p) == want, (flags, tun)
        pe = xm.Plan(pat, xm.XM_INDUCED | xm.XM_EMBEDDINGS)
        assert xm.xm_count(g, pe) == og.count_embeddings(pat, induced=True)
    g, og = tiny
    p = xm.Plan(pat, xm.XM_INDUCED)
    want = og.count_matches(pat, induced=True)
    out = torch.full((max(want, 1) * pat[0],), -1, dtype=torch.int32, device="cuda")
    total, written, over = xm.xm_enumerate(g, p, out)
    assert total == want == written
    rows = oracle.canonicalize(pat, out[: want * pat[0]].view(-1, pat[0]).cpu().numpy())
    assert np.array_equal(rows, og.enumerate(pat, induced=True))


def test_induced_motif_census_s20(xm, s20):
    """Full scale-20 graph, no oracle needed: the induced counts of the 13
    motifs follow from the non-induced counts through the exact (integer,
    unitriangular) motif containment matrix, and they partition the weakly
    connected node triples; spot-checked per start node against the oracle."""
    g, og = s20
    names = list(synth.MOTIFS3)
    C = np.zeros((13, 13), dtype=object)
    for j, nj in enumerate(names):
        k, arcs = synth.MOTIFS3[nj]
        small = oracle.OracleGraph(3, np.array([a for a, _ in arcs], np.int32),
                                   np.array([b for _, b in arcs], np.int32))
        for i, ni in enumerate(names):
            C[i, j] = small.count_matches(synth.MOTIFS3[ni])
    plain = np.array([xm.xm_count(g, xm.Plan(synth.MOTIFS3[nm])) for nm in names], dtype=object)
    induced = np.array([xm.xm_count(g, xm.Plan(synth.MOTIFS3[nm], xm.XM_INDUCED)) for nm in names], dtype=object)
    assert list(C.dot(induced)) == list(plain)
    rng = np.random.default_rng(21)
    for nm in names:
        pe = xm.Plan(synth.MOTIFS3[nm], xm.XM_INDUCED | xm.XM_EMBEDDINGS)
        for v in rng.integers(0, og.n, 6):
            v = int(v)
            assert xm.xm_count_range(g, pe, v, v + 1) == og.count_embeddings(synth.MOTIFS3[nm], pe.start, v, v + 1,
                                                                             induced=True)


def test_plan_autotuner(xm, rmat_small):
    g, og = rmat_small
    p = xm.Plan(synth.BIFAN)
    want = og.count_matches(synth.BIFAN)
    cands = [(64, 1, 2, 0, 0), (256, 8, 8, 0, 0), (512, 32, 4, 1, 0)]
    best, ms = xm.xm_plan_tune(g, p, cands, reps=2)
    assert ms > 0 and tuple(best.values())[:5] in cands and best["merge_ratio"] == 2
    assert p.tuning() == best
    assert xm.xm_count(g, p) == want
    # on a start-node list, with the intersection strategy as a knob
    roots = np.arange(0, g.n, 3, dtype=np.int32)
    want_roots = xm.xm_count_roots(g, p, roots)
    cands = [(64, 1, 2, 0, 0, -1), (256, 8, 8, 0, 0, 8), (512, 32, 4, 1, 0, 1024)]
    best, ms = xm.xm_plan_tune(g, p, cands, reps=2, roots=roots)
    assert ms > 0 and tuple(best.values()) in cands
    assert xm.xm_count_roots(g, p, roots) == want_roots


# ------------------------------------------------ leaf products (Sec. 5.3)

PRODUCT_PATTERNS = {
    "star4": (4, [(0, 1), (0, 2), (0, 3)]),
    "instar4": (4, [(1, 0), (2, 0), (3, 0)]),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "mixstar": (4, [(0, 1), (2, 0), (0, 3)]),
    "star5": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
    "tri_tail": (5, [(0, 1), (1, 2), (0, 2), (2, 3), (2, 4)]),
    "recip_star": (5, [(0, 1), (1, 0), (0, 2), (2, 0), (0, 3), (0, 4)]),
    "fan3": (5, [(0, 1), (0, 2), (0, 3), (4, 1), (4, 2), (4, 3)]),
    "path5": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "ffchain5": synth.FFCHAIN5,
}


@pytest.mark.parametrize("name", sorted(PRODUCT_PATTERNS))
def test_products_tiny(xm, tiny, name):
    """Counting with a leaf product (choose or inclusion-exclusion) equals
    the oracle and the plain level-by-level walk, in every plan variant."""
    g, og = tiny
    pat = PRODUCT_PATTERNS[name]
    want = og.count_matches(pat)
    assert xm.Plan(pat).product()["r"] > 0
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE, xm.XM_NO_PRODUCT):
        for tun in TUNINGS:
            p = xm.Plan(pat, flags)
            p.set_tuning(**tun)
            assert xm.xm_count(g, p) == want, (flags, tun)
    assert xm.xm_count(g, xm.Plan(pat, xm.XM_EMBEDDINGS)) == og.count_embeddings(pat)


@pytest.mark.parametrize("name", ["star4", "instar4", "path4", "mixstar", "tri_tail", "recip_star", "fan3",
                                  "path5", "ffchain5"])
def test_products_rmat(xm, rmat_tiny, name):
    g, og = rmat_tiny
    pat = PRODUCT_PATTERNS[name]
    want = og.count_matches(pat)
    for tun in (TUNINGS[0], TUNINGS[2]):
        p = xm.Plan(pat)
        p.set_tuning(**tun)
        assert xm.xm_count(g, p) == want, tun
    assert xm.xm_count(g, xm.Plan(pat, xm.XM_NO_PRODUCT)) == want
    c, st = xm.xm_count_stats(g, xm.Plan(pat))
    assert c == want and st["alg_bytes"] > 0


def test_products_root_ranges_and_enumeration(xm, tiny, rmat_tiny):
    g, og = rmat_tiny
    for name in ("path4", "mixstar", "ffchain5"):
        pat = PRODUCT_PATTERNS[name]
        p = xm.Plan(pat)
        whole = xm.xm_count(g, p)
        cuts = [0, 1, 3, 100, 257, g.n]
        assert sum(xm.xm_count_range(g, p, a, b) for a, b in zip(cuts, cuts[1:])) == whole
        pe = xm.Plan(pat, xm.XM_EMBEDDINGS)
        for r in (0, 1, 7, 300):
            assert xm.xm_count_range(g, pe, r, r + 1) == og.count_embeddings(pat, pe.start, r, r + 1)
    # enumeration walks every level; the plan's reordered vertices still
    # land in pattern-vertex order
    g, og = tiny
    for name in ("path4", "tri_tail", "star4"):
        pat = PRODUCT_PATTERNS[name]
        want = og.count_matches(pat)
        p = xm.Plan(pat)
        out = torch.full((max(want, 1) * pat[0],), -1, dtype=torch.int32, device="cuda")
        total, written, over = xm.xm_enumerate(g, p, out)
        assert total == want and written == want and not over
        rows = oracle.canonicalize(pat, out[: want * pat[0]].view(-1, pat[0]).cpu().numpy())
        assert np.array_equal(rows, og.enumerate(pat))


def test_product_stars_s20_beyond_64_bits(xm, s20):
    """Out- and in-stars at full size against exact closed forms: a star with
    r leaves has sum_v C(outdeg(v), r) matches. The six-leaf out-star sums
    past 2^64, through the 128-bit product path."""
    from math import comb
    g, og = s20
    off, adj = og.out_csr()
    outdeg = np.diff(off)
    indeg = np.bincount(adj, minlength=og.n)
    for r, deg, inward in ((3, outdeg, False), (4, indeg, True), (6, outdeg, False)):
        arcs = [(i, 0) for i in range(1, r + 1)] if inward else [(0, i) for i in range(1, r + 1)]
        pat = (r + 1, arcs)
        p = xm.Plan(pat)
        assert p.product()["kind"] == xm.XM_PROD_CHOOSE
        vals, cnts = np.unique(deg, return_counts=True)
        want = sum(comb(int(d), r) * int(c) for d, c in zip(vals, cnts))
        got = xm.xm_count(g, p)
        assert got == want, r
        if r == 6:
            assert want > 2 ** 64


# ------------------------------------------ cut-vertex decomposition (count)

SPLIT_PATTERNS = {
    "ffchain5": synth.FFCHAIN5,
    "path5": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "tri_tail": (5, [(0, 1), (1, 2), (0, 2), (2, 3), (2, 4)]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
    "four_parts": (6, [(0, 1), (1, 0), (0, 2), (2, 3), (3, 0), (4, 0), (0, 5)]),
    "recip_path": (5, [(0, 1), (1, 0), (1, 2), (2, 3), (3, 2), (3, 4)]),
}


@pytest.mark.parametrize("name", ["path8", "spider8", "double_star8"])
def test_split_counts_eight_vertices(xm, name):
    """Eight-vertex patterns whose splits have dozens of quotient classes,
    themselves split again, on a sparse ER graph the oracle walks quickly."""
    pat = {"path8": (8, [(i, i + 1) for i in range(7)]),
           "spider8": (8, [(1, 0), (2, 1), (3, 0), (4, 3), (0, 5), (5, 6), (7, 0)]),
           "double_star8": (8, [(0, 1), (0, 2), (0, 3), (0, 4), (4, 5), (4, 6), (4, 7)])}[name]
    n, src, dst = synth.er_graph(300, 900, seed=9)
    g, og = graph_pair(xm, n, src, dst)
    assert xm.Plan(pat).split()["cut"] >= 0
    want = og.count_matches(pat)
    assert want > 0
    for flags in (xm.XM_REDUCE, xm.XM_NO_SPLIT, xm.XM_NO_PRODUCT | xm.XM_NO_REDUCE):
        assert xm.xm_count(g, xm.Plan(pat, flags)) == want, flags
    assert xm.xm_count(g, xm.Plan(pat, xm.XM_EMBEDDINGS)) == og.count_embeddings(pat)


@pytest.mark.parametrize("name", ["ffchain5", "tri_tail", "bowtie", "path5"])
def test_split_over_start_node_subsets(xm, rmat_small, name):
    """Counts over start-node ranges and lists through the cut-vertex split
    rooted at the start vertex (part counts per start node, their product
    sum, rooted quotients) equal the whole-pattern walk over the same start
    nodes and the oracle rooted at the start vertex; ranges that partition
    the nodes add up to xm_count; the instrumented count agrees; a pattern
    whose cut vertex is not its start vertex (path5) is walked."""
    g, og = rmat_small
    pat = SPLIT_PATTERNS[name]
    p, walk = xm.Plan(pat), xm.Plan(pat, xm.XM_NO_SPLIT)
    pe, walk_e = xm.Plan(pat, xm.XM_EMBEDDINGS), xm.Plan(pat, xm.XM_EMBEDDINGS | xm.XM_NO_SPLIT)
    assert p.split()["cut"] >= 0
    cuts = [0, 1, 3, 64, 500, 900, g.n]
    per = [xm.xm_count_range(g, p, a, b) for a, b in zip(cuts, cuts[1:])]
    assert per == [xm.xm_count_range(g, walk, a, b) for a, b in zip(cuts, cuts[1:])]
    assert sum(per) == xm.xm_count(g, p) == og.count_matches(pat)
    prep, match = g.last_timing()
    assert prep >= 0 and match > 0
    rng = np.random.default_rng(11)
    # the hubs of the skewed graph and a seeded uniform sample
    off, adj = og.out_csr()
    deg = np.diff(off) + np.bincount(adj, minlength=g.n)
    roots = np.concatenate([np.argsort(-deg)[:6], rng.integers(0, g.n, 30)]).astype(np.int32)
    want = [og.count_embeddings(pat, pe.start, v, v + 1) for v in roots.tolist()]
    assert xm.xm_count_roots_each(g, pe, roots) == want
    assert xm.xm_count_roots_each(g, walk_e, roots) == want
    uniq = np.unique(roots)
    c = xm.xm_count_roots(g, p, uniq)
    assert c == xm.xm_count_roots(g, walk, uniq) == sum(xm.xm_count_roots_each(g, p, uniq))
    assert xm.xm_count_roots(g, pe, uniq) == sum(og.count_embeddings(pat, pe.start, v, v + 1) for v in uniq.tolist())
    cs, st = xm.xm_count_roots_stats(g, p, uniq)
    assert cs == c and st["alg_bytes"] > 0
    cs, st = xm.xm_count_stats(g, p, 64, 500)
    assert cs == per[3] and st["alg_bytes"] > 0


@pytest.mark.parametrize("name", sorted(SPLIT_PATTERNS))
def test_split_counts(xm, tiny, rmat_tiny, name):
    """xm_count through the cut-vertex decomposition (per-node part counts,
    product sum, quotient counts) equals the oracle and the whole-pattern
    walk."""
    pat = SPLIT_PATTERNS[name]
    assert xm.Plan(pat).split()["cut"] >= 0
    # the six-vertex pattern takes the oracle minutes on the skewed graph
    for g, og in ((tiny,) if name == "four_parts" else (tiny, rmat_tiny)):
        want = og.count_matches(pat)
        for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE, xm.XM_NO_SPLIT, xm.XM_NO_PRODUCT):
            for tun in (TUNINGS[0], TUNINGS[1]):
                p = xm.Plan(pat, flags)
                p.set_tuning(**tun)
                assert xm.xm_count(g, p) == want, (flags, tun)
        assert xm.xm_count(g, xm.Plan(pat, xm.XM_EMBEDDINGS)) == og.count_embeddings(pat)
