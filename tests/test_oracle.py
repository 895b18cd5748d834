"""Pins for the CPU oracle, independent of the oracle's own code.

Each check ties the oracle to something it does not compute itself:
  * brute force over every node k-tuple on tiny graphs (embeddings, and
    distinct matched subgraphs identified by their image arc sets -- the
    problem statement of Sec. 2, without any orbit arithmetic);
  * closed forms from adjacency-matrix algebra (directed 3-cycles tr(A^3)/3,
    feed-forward triangles sum(A o A^2), bi-fan, bi-parallel, directed
    4-cycle, stars and 2-paths) on seeded random digraphs;
  * counts on complete digraphs derived by hand;
  * invariants: arc reversal, node relabelling, root-range additivity,
    #embeddings = |Aut(P)| * #matches.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth


# ------------------------------------------------------------ helpers --

def simple_arcs(n, src, dst):
    """Distinct arcs without self-loops, as a Python set (the data graph of Def. 2.1)."""
    return {(int(u), int(v)) for u, v in zip(src, dst) if u != v}


def brute_force(n, arcs, pattern):
    """(#embeddings, set of image arc sets) over all k-tuples of nodes."""
    k, parcs = pattern
    emb = 0
    images = set()
    for t in itertools.product(range(n), repeat=k):
        if len(set(t)) != k:
            continue
        if all((t[u], t[v]) in arcs for u, v in parcs):
            emb += 1
            images.add(frozenset((t[u], t[v]) for u, v in parcs))
    return emb, images


def random_small_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    u, v = np.nonzero(a)
    return n, u.astype(np.int32), v.astype(np.int32)


def adjacency(n, src, dst):
    arcs = simple_arcs(n, src, dst)
    r = np.array([a for a, _ in arcs], np.int64)
    c = np.array([b for _, b in arcs], np.int64)
    return sp.csr_matrix((np.ones(len(arcs), np.int64), (r, c)), shape=(n, n))


def transpose_pattern(pattern):
    k, arcs = pattern
    return k, [(b, a) for a, b in arcs]


SMALL_PATTERNS = [synth.CYCLE3, synth.FFL, synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL,
                  (3, [(0, 1), (1, 0), (1, 2)]),              # reciprocal pair + arc
                  (3, [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]),  # complete digraph
                  (2, [(0, 1)]), (2, [(0, 1), (1, 0)]),
                  (4, [(0, 1), (1, 2), (2, 0), (2, 3)])]     # triangle with a tail


def brute_aut(pattern):
    k, arcs = pattern
    s = set(arcs)
    return sum(1 for p in itertools.permutations(range(k))
               if {(p[a], p[b]) for a, b in arcs} == s)


# --------------------------------------------------------- brute force --

@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("pattern", SMALL_PATTERNS)
def test_oracle_vs_brute_force(seed, pattern):
    n, src, dst = random_small_graph(8, 0.4, seed)
    # add a repeated arc and a self-loop: the oracle must drop them
    src = np.concatenate([src, src[:1], np.array([3], np.int32)])
    dst = np.concatenate([dst, dst[:1], np.array([3], np.int32)])
    arcs = simple_arcs(n, src, dst)
    emb, images = brute_force(n, arcs, pattern)
    g = oracle.OracleGraph(n, src, dst)
    assert g.m == len(arcs)
    assert g.count_embeddings(pattern) == emb
    assert g.count_matches(pattern) == len(images)
    rows = g.enumerate(pattern)
    assert rows.shape[0] == len(images)
    k, parcs = pattern
    got = {frozenset((int(r[u]), int(r[v])) for u, v in parcs) for r in rows}
    assert got == images
    # each row is an embedding and the orbit-smallest one
    assert np.array_equal(oracle.canonicalize(pattern, rows), rows)


@pytest.mark.parametrize("pattern", [synth.FFCHAIN5, (5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)])])
def test_oracle_five_vertices_brute_force(pattern):
    n, src, dst = random_small_graph(7, 0.55, 11)
    arcs = simple_arcs(n, src, dst)
    emb, images = brute_force(n, arcs, pattern)
    g = oracle.OracleGraph(n, src, dst)
    assert g.count_embeddings(pattern) == emb
    assert g.count_matches(pattern) == len(images)


@pytest.mark.parametrize("pattern", SMALL_PATTERNS + [synth.FFCHAIN5] + list(synth.MOTIFS3.values()))
def test_aut_sizes(pattern):
    aut = oracle.automorphisms(pattern)
    assert aut.shape[0] == brute_aut(pattern)
    # every row is a permutation
    for row in aut:
        assert sorted(row.tolist()) == list(range(pattern[0]))


def test_named_aut_sizes():
    # |Aut| of the named workloads, derived by hand from their arc lists
    assert oracle.automorphisms(synth.CYCLE3).shape[0] == 3
    assert oracle.automorphisms(synth.FFL).shape[0] == 1
    assert oracle.automorphisms(synth.BIFAN).shape[0] == 4
    assert oracle.automorphisms(synth.CYCLE4).shape[0] == 4
    assert oracle.automorphisms(synth.BIPARALLEL).shape[0] == 2
    assert oracle.automorphisms(synth.FFCHAIN5).shape[0] == 2


# --------------------------------------------------------- closed forms --

def closed_forms(n, src, dst):
    A = adjacency(n, src, dst)
    AT = A.T.tocsr()
    A2 = (A @ A).tocsr()
    outdeg = np.asarray(A.sum(axis=1)).ravel()
    indeg = np.asarray(A.sum(axis=0)).ravel()
    r = np.asarray(A.multiply(AT).sum(axis=1)).ravel()          # reciprocal partners
    res = {}
    res["cycle3"] = int(A2.multiply(AT).sum()) // 3              # tr(A^3) / 3
    res["ffl"] = int(A.multiply(A2).sum())                       # sum(A o A^2)
    ata = sp.triu(AT @ A, k=1).tocoo()                           # |in(c) & in(d)|, c < d
    res["bifan"] = int((ata.data * (ata.data - 1) // 2).sum())
    aat = sp.triu(A @ AT, k=1).tocoo()                           # |out(a) & out(b)|, a < b
    res["bifan_by_sources"] = int((aat.data * (aat.data - 1) // 2).sum())
    a2 = A2.tocoo()
    off = a2.row != a2.col
    res["biparallel"] = int((a2.data[off] * (a2.data[off] - 1) // 2).sum())
    tr4 = int(A2.multiply(A2.T).sum())                           # tr(A^4)
    res["cycle4"] = (tr4 - 2 * int((r * r).sum()) + int(r.sum())) // 4
    res["outstar"] = int((outdeg * (outdeg - 1) // 2).sum())
    res["instar"] = int((indeg * (indeg - 1) // 2).sum())
    res["path2"] = int((indeg * outdeg - r).sum())
    return res


CF_PATTERNS = {"cycle3": synth.CYCLE3, "ffl": synth.FFL, "bifan": synth.BIFAN,
               "biparallel": synth.BIPARALLEL, "cycle4": synth.CYCLE4,
               "outstar": synth.MOTIFS3["021D"], "instar": synth.MOTIFS3["021U"],
               "path2": synth.MOTIFS3["021C"]}


def test_closed_forms_match_brute_force():
    # the closed forms themselves, checked by brute force on small graphs
    for seed in range(4):
        n, src, dst = random_small_graph(9, 0.35, 100 + seed)
        cf = closed_forms(n, src, dst)
        arcs = simple_arcs(n, src, dst)
        assert cf["bifan"] == cf["bifan_by_sources"]
        for name, pat in CF_PATTERNS.items():
            if pat[0] <= 4:
                _, images = brute_force(n, arcs, pat)
                assert cf[name] == len(images), name


@pytest.mark.parametrize("which", ["tiny_er", "rmat10"])
def test_oracle_vs_closed_forms(which):
    if which == "tiny_er":
        n, src, dst = synth.tiny_er()
    else:
        n, src, dst = synth.rmat_graph(10, 8, seed=7)
    g = oracle.OracleGraph(n, src, dst)
    cf = closed_forms(n, src, dst)
    assert cf["bifan"] == cf["bifan_by_sources"]
    for name, pat in CF_PATTERNS.items():
        assert g.count_matches(pat) == cf[name], name


def test_complete_digraph_counts():
    # complete digraph on n nodes: every ordered pair is an arc
    n = 7
    src, dst = zip(*[(u, v) for u in range(n) for v in range(n) if u != v])
    g = oracle.OracleGraph(n, np.array(src, np.int32), np.array(dst, np.int32))
    c = math.comb
    assert g.count_matches(synth.CYCLE3) == 2 * c(n, 3)           # two cyclic orientations per triple
    assert g.count_matches(synth.FFL) == 6 * c(n, 3)              # 3! transitive orders per triple
    assert g.count_matches(synth.CYCLE4) == 6 * c(n, 4)           # (4-1)! cyclic orders per 4-set
    assert g.count_matches(synth.BIFAN) == c(n, 2) * c(n - 2, 2)  # sources pair, sinks pair
    assert g.count_matches(synth.BIPARALLEL) == n * (n - 1) * c(n - 2, 2)
    assert g.count_embeddings(synth.CYCLE3) == n * (n - 1) * (n - 2)


# ------------------------------------------------------------ invariants --

@pytest.mark.parametrize("pattern", [synth.FFL, synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL, synth.FFCHAIN5])
def test_invariants(pattern):
    n, src, dst = synth.er_graph(300, 2400, seed=21)
    g = oracle.OracleGraph(n, src, dst)
    matches = g.count_matches(pattern)
    emb = g.count_embeddings(pattern)
    assert emb == oracle.automorphisms(pattern).shape[0] * matches
    # arc reversal: count(P, G) == count(P^T, G^T)
    gt = oracle.OracleGraph(n, dst, src)
    assert gt.count_matches(transpose_pattern(pattern)) == matches
    # node relabelling
    perm = np.random.default_rng(5).permutation(n).astype(np.int32)
    gp = oracle.OracleGraph(n, perm[src], perm[dst])
    assert gp.count_matches(pattern) == matches
    # root-range additivity, for every choice of root vertex
    for root in range(pattern[0]):
        cuts = [0, 37, 150, 151, n]
        parts = sum(g.count_embeddings(pattern, root, a, b) for a, b in zip(cuts, cuts[1:]))
        assert parts == emb


def test_motifs3_are_the_13_classes():
    # all labelled digraphs on 3 nodes, weakly connected, up to isomorphism
    pairs = [(u, v) for u in range(3) for v in range(3) if u != v]

    def canon(arcs):
        return min(tuple(sorted((p[a], p[b]) for a, b in arcs)) for p in itertools.permutations(range(3)))

    classes = set()
    for mask in range(1, 64):
        arcs = [pairs[i] for i in range(6) if mask >> i & 1]
        touched = {x for a in arcs for x in a}
        und = {frozenset(a) for a in arcs}
        if len(touched) == 3 and len(und) >= 2:
            classes.add(canon(arcs))
    assert len(classes) == 13
    assert {canon(p[1]) for p in synth.MOTIFS3.values()} == classes


def test_synth_is_deterministic():
    a = synth.rmat_graph(12, 4, seed=9)
    b = synth.rmat_graph(12, 4, seed=9)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    n, src, dst = synth.tiny_er()
    assert n == 2000 and len(src) == 20000
    assert len({(int(u), int(v)) for u, v in zip(src, dst)}) == 20000
    assert not np.any(src == dst)


# ------------------------------------------------------ induced variant --

def brute_force_induced(n, arcs, pattern):
    """(#embeddings, set of image node sets): every ordered pair of pattern
    vertices is an arc of the pattern iff its image is an arc of G."""
    k, parcs = pattern
    pset = set(parcs)
    emb = 0
    images = set()
    for t in itertools.product(range(n), repeat=k):
        if len(set(t)) != k:
            continue
        if all(((t[u], t[v]) in arcs) == ((u, v) in pset) for u in range(k) for v in range(k) if u != v):
            emb += 1
            images.add(frozenset(t))
    return emb, images


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("pattern", SMALL_PATTERNS + [synth.FFCHAIN5])
def test_induced_oracle_vs_brute_force(seed, pattern):
    n, src, dst = random_small_graph(7 if pattern[0] <= 4 else 6, 0.45, 50 + seed)
    arcs = simple_arcs(n, src, dst)
    emb, images = brute_force_induced(n, arcs, pattern)
    g = oracle.OracleGraph(n, src, dst)
    assert g.count_embeddings(pattern, induced=True) == emb
    assert g.count_matches(pattern, induced=True) == len(images)
    rows = g.enumerate(pattern, induced=True)
    assert {frozenset(int(x) for x in r) for r in rows} == images


def motif_containment():
    """C[i][j] = non-induced matches of motif i inside motif j (as a graph)."""
    names = list(synth.MOTIFS3)
    C = np.zeros((13, 13), dtype=object)
    for j, nj in enumerate(names):
        k, arcs = synth.MOTIFS3[nj]
        g = oracle.OracleGraph(3, np.array([a for a, _ in arcs], np.int32), np.array([b for _, b in arcs], np.int32))
        for i, ni in enumerate(names):
            C[i, j] = g.count_matches(synth.MOTIFS3[ni])
    return names, C


def test_motif_census_identities():
    # induced counts of the 13 classes partition the weakly connected node
    # triples; non-induced counts follow from them through the containment
    # matrix (unitriangular once motifs are sorted by arc count)
    names, C = motif_containment()
    assert all(C[i, i] == 1 for i in range(13))
    order = sorted(range(13), key=lambda i: len(synth.MOTIFS3[names[i]][1]))
    for a in range(13):
        for b in range(a):
            assert C[order[a], order[b]] == 0  # a sparser motif never contains a denser one
    n, src, dst = random_small_graph(11, 0.3, 9)
    arcs = simple_arcs(n, src, dst)
    und = {frozenset(a) for a in arcs}
    connected_triples = 0
    for t in itertools.combinations(range(n), 3):
        pairs = [frozenset((t[i], t[j])) for i in range(3) for j in range(i + 1, 3)]
        if sum(p in und for p in pairs) >= 2:
            connected_triples += 1
    g = oracle.OracleGraph(n, src, dst)
    induced = np.array([g.count_matches(synth.MOTIFS3[nm], induced=True) for nm in names], dtype=object)
    plain = np.array([g.count_matches(synth.MOTIFS3[nm]) for nm in names], dtype=object)
    assert sum(induced) == connected_triples
    assert list(C.dot(induced)) == list(plain)


# ------------------------------------------- rooted enumeration, triangles --

@pytest.mark.parametrize("pattern", [synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL, synth.FFL,
                                     (4, [(0, 1), (1, 2), (2, 0), (2, 3)])])
def test_enumerate_embeddings_vs_brute_force(pattern):
    """Every embedding with the root vertex's node in a range, against all
    node k-tuples."""
    n, src, dst = random_small_graph(8, 0.45, 31)
    arcs = simple_arcs(n, src, dst)
    k, parcs = pattern
    g = oracle.OracleGraph(n, src, dst)
    for root, lo, hi in ((0, 0, n), (1, 2, 5), (k - 1, 6, 7), (0, 3, 3)):
        want = sorted(t for t in itertools.product(range(n), repeat=k)
                      if len(set(t)) == k and lo <= t[root] < hi and all((t[u], t[v]) in arcs for u, v in parcs))
        got = g.enumerate_embeddings(pattern, root, lo, hi)
        assert [tuple(r) for r in got.tolist()] == want
        assert g.count_embeddings(pattern, root, lo, hi) == len(want)


def test_triangle_sums_vs_brute_force_and_matrices():
    """Feed-forward triangles and closed 3-walks per source range against
    brute force over node triples (tiny graphs) and sparse matrix products
    (R-MAT scale 10); additive over a partition of the sources."""
    for seed in (0, 1):
        n, src, dst = random_small_graph(9, 0.4, 40 + seed)
        arcs = simple_arcs(n, src, dst)
        ffl = sum(1 for a, b, c in itertools.permutations(range(n), 3)
                  if (a, b) in arcs and (b, c) in arcs and (a, c) in arcs)
        walks = sum(1 for a, b, c in itertools.permutations(range(n), 3)
                    if (a, b) in arcs and (b, c) in arcs and (c, a) in arcs)
        g = oracle.OracleGraph(n, src, dst)
        assert g.triangle_sums() == (ffl, walks)
    n, src, dst = synth.rmat_graph(10, 6, seed=17)
    A = adjacency(n, src, dst)
    A2 = A @ A
    g = oracle.OracleGraph(n, src, dst)
    f, c = g.triangle_sums()
    assert f == int(A.multiply(A2).sum())
    assert c == int((A2 @ A).diagonal().sum())
    assert f == g.count_matches(synth.FFL) and c == 3 * g.count_matches(synth.CYCLE3)
    cuts = [0, 1, 7, 300, n]
    parts = [g.triangle_sums(a, b) for a, b in zip(cuts, cuts[1:])]
    assert (sum(p[0] for p in parts), sum(p[1] for p in parts)) == (f, c)


@pytest.mark.parametrize("pattern", [synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL, synth.FFCHAIN5,
                                     synth.MOTIFS3["300"], synth.MOTIFS3["201"]])
def test_canonicalize_restores_orbit_minimum(pattern):
    """Each orbit-smallest row, moved by a random automorphism (a different
    embedding of the same match whenever the automorphism moves a vertex),
    is mapped back to the row itself."""
    n, src, dst = random_small_graph(9, 0.7, 5)
    g = oracle.OracleGraph(n, src, dst)
    rows = g.enumerate(pattern)
    assert rows.shape[0] > 0
    aut = oracle.automorphisms(pattern)
    rng = np.random.default_rng(9)
    pick = aut[rng.integers(0, aut.shape[0], rows.shape[0])]
    moved = np.take_along_axis(rows, pick, axis=1)        # moved[i][v] = rows[i][s(v)]
    if aut.shape[0] > 1:
        assert not np.array_equal(moved, rows)
    assert np.array_equal(oracle.canonicalize(pattern, moved), rows)
    # every embedding of the match canonicalises to the same row
    for s in aut:
        assert np.array_equal(oracle.canonicalize(pattern, rows[:, s]), rows)


def test_capped_walk_counts_or_gives_up():
    """The capped walk returns the exact rooted count whenever it finishes
    within its candidate budget, gives up (None) below the work the walk
    needs, and finishes for every root once the cap is large."""
    n, src, dst = synth.rmat_graph(9, 8, seed=17)
    g = oracle.OracleGraph(n, src, dst)
    for pat in (synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5):
        gave_up = 0
        for v in range(0, n, 17):
            want = g.count_embeddings(pat, 0, v, v + 1)
            assert g.count_embeddings_capped(pat, 0, v, v + 1, 1 << 40) == want
            got = g.count_embeddings_capped(pat, 0, v, v + 1, 50)
            assert got is None or got == want
            gave_up += got is None
        assert gave_up > 0
    # cap 1: only walks that examine at most one candidate finish
    assert g.count_embeddings_capped(synth.BIFAN, 0, 0, 1, 1) is None
