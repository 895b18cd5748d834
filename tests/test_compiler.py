"""Host-side checks of the C-ABI library: symbol exports, pattern compiler
(Sec. 4 reduction, Sec. 5.1 plan, symmetry conditions), and the plan IR's
meaning, executed by a slow CPU interpreter against the oracle."""
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2404_11105_b300 as xm
from tests.plan_interp import adjacency_lists, run_plan

HEADER = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "include", "xm.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(xm_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol():
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(xm.lib(), s), s
    assert set(syms) == set(xm.EXPORTS)
    assert xm.lib().xm_version() >= 100
    assert xm.lib().xm_strerror(3) == b"XM_EOVERFLOW"


@pytest.mark.parametrize("bad", [
    (3, [(0, 0), (0, 1), (1, 2)]),            # self-loop
    (3, [(0, 1), (0, 1), (1, 2)]),            # repeated arc
    (4, [(0, 1), (2, 3)]),                    # not weakly connected
    (9, [(i, i + 1) for i in range(8)]),      # k > 8
    (3, [(0, 1), (1, 5)]),                    # id out of range
])
def test_compile_rejects_bad_patterns(bad):
    with pytest.raises(xm.XmError) as ei:
        xm.Plan(bad)
    assert ei.value.status == xm.XM_EINVAL


def random_patterns(count, seed):
    pats = []
    for i in range(count):
        u = synth.uniforms(seed, 1000 + i, 2)
        k = 3 + int(u[0] * 4)              # 3..6
        rho = 0.3 + 0.4 * u[1]
        pats.append(synth.random_pattern(k, rho, seed, i))
    return pats


NAMED = [synth.CYCLE3, synth.FFL, synth.BIFAN, synth.CYCLE4, synth.BIPARALLEL, synth.FFCHAIN5]


@pytest.mark.parametrize("pattern", NAMED + list(synth.MOTIFS3.values()) + random_patterns(12, 77))
def test_plan_structure(pattern):
    k, arcs = pattern
    aset = set(arcs)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE, xm.XM_EMBEDDINGS):
        p = xm.Plan(pattern, flags)
        assert p.k == k and p.n_levels == k
        assert p.aut_size == oracle.automorphisms(pattern).shape[0]
        order = p.order()
        assert sorted(order) == list(range(k))
        assert order[0] == p.start
        # Alg. 1 starts at a vertex of maximal degree
        deg = [sum(1 for a in arcs if v in a) for v in range(k)]
        assert deg[p.start] == max(deg)
        if flags & xm.XM_NO_REDUCE:
            assert p.n_reuse == 0
        for l in range(k):
            L = p.level(l)
            assert L["vertex"] == order[l]
            v = order[l]
            want = sorted([(j, 0) for j in range(l) if (order[j], v) in aset] +
                          [(j, 1) for j in range(l) if (v, order[j]) in aset])
            assert sorted(L["ops"]) == want
            if l > 0:
                assert L["ops"], "every later level hangs off an earlier one"
            # degree thresholds never exceed the pattern degrees (weakened on
            # reuse sources, dropped where the operand lists imply them)
            dout = sum(1 for a, _ in arcs if a == v)
            din = sum(1 for _, b in arcs if b == v)
            nout = sum(1 for _, d in L["ops"] if d == 0)
            nin = sum(1 for _, d in L["ops"] if d == 1)
            assert L["dout_min"] <= dout and L["din_min"] <= din
            if not any(p.level(q)["reuse"] == l for q in range(l + 1, k)):
                assert L["dout_min"] == (dout if dout > nin else 0)
                assert L["din_min"] == (din if din > nout else 0)
            if L["reuse"] >= 0:
                R = p.level(L["reuse"])
                assert 1 <= L["reuse"] < l
                assert set(R["ops"]) <= set(L["ops"])
            if flags & xm.XM_EMBEDDINGS:
                assert L["lo_mask"] == 0 and L["hi_mask"] == 0


def test_loops_are_not_reduced():
    # 3_p and 4_p are loops whose vertices and edges are equivalent: no reduction (Sec. 6.3)
    assert xm.Plan(synth.CYCLE3).n_reuse == 0
    assert xm.Plan(synth.CYCLE4).n_reuse == 0


def test_shared_endpoints_are_reduced():
    # edges sharing a source or destination include each other (Thm. 2.1): reuse appears
    assert xm.Plan(synth.FFL).n_reuse >= 1
    assert xm.Plan(synth.BIFAN).n_reuse >= 1
    assert xm.Plan(synth.MOTIFS3["021D"]).n_reuse >= 1
    assert "split:" in xm.Plan(synth.BIFAN).describe()


def test_tuning_roundtrip_and_validation():
    p = xm.Plan(synth.BIFAN)
    p.set_tuning(window=256, unit=16, warps_per_block=4, blocks_per_sm=2)
    # merge_ratio 0 resolves to the default length ratio (2)
    assert p.tuning() == {"window": 256, "unit": 16, "warps_per_block": 4, "blocks_per_sm": 2, "budget_ms": 0,
                          "merge_ratio": 2}
    p.set_tuning(merge_ratio=-1)
    assert p.tuning()["merge_ratio"] == -1
    p.set_tuning(merge_ratio=1024)
    assert p.tuning()["merge_ratio"] == 1024
    for bad in (dict(window=100), dict(merge_ratio=-2), dict(merge_ratio=1025)):
        with pytest.raises(xm.XmError):
            p.set_tuning(**bad)
    assert p.tuning()["merge_ratio"] == 1024


DENSE = [synth.random_pattern(k, 0.9, 123, k) for k in (6, 7, 8)] + \
        [(8, [(u, v) for u in range(8) for v in range(8) if u != v])]


@pytest.mark.parametrize("pattern", DENSE)
def test_dense_patterns_use_many_operands(pattern):
    # a vertex with arcs both ways to every earlier vertex has 2(k-1) operands
    k = pattern[0]
    p = xm.Plan(pattern)
    assert max(len(p.level(l)["ops"]) for l in range(k)) > 7
    n, src, dst = synth.er_graph(12, 100, seed=2)
    out, inn = adjacency_lists(n, src, dst)
    g = oracle.OracleGraph(n, src, dst)
    assert run_plan(n, out, inn, p) == g.count_matches(pattern)
    assert run_plan(n, out, inn, xm.Plan(pattern, xm.XM_NO_REDUCE)) == g.count_matches(pattern)


@pytest.mark.parametrize("seed", [3, 4])
@pytest.mark.parametrize("pattern", NAMED + list(synth.MOTIFS3.values()) + random_patterns(10, 91))
def test_plan_semantics_vs_oracle(seed, pattern):
    k = pattern[0]
    n, src, dst = synth.er_graph(11 if k <= 4 else 9, 50 if k <= 4 else 40, seed=seed)
    out, inn = adjacency_lists(n, src, dst)
    g = oracle.OracleGraph(n, src, dst)
    want = g.count_matches(pattern)
    want_emb = g.count_embeddings(pattern)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE):
        p = xm.Plan(pattern, flags)
        assert run_plan(n, out, inn, p, use_reuse=True) == want
        assert run_plan(n, out, inn, p, use_reuse=False) == want
    pe = xm.Plan(pattern, xm.XM_EMBEDDINGS)
    assert run_plan(n, out, inn, pe) == want_emb


@pytest.mark.parametrize("pattern", NAMED + list(synth.MOTIFS3.values()) + random_patterns(8, 17))
def test_induced_plans_vs_oracle(pattern):
    k, arcs = pattern
    aset = set(arcs)
    n, src, dst = synth.er_graph(10, 40, seed=8)
    out, inn = adjacency_lists(n, src, dst)
    g = oracle.OracleGraph(n, src, dst)
    for flags in (xm.XM_INDUCED, xm.XM_INDUCED | xm.XM_NO_REDUCE):
        p = xm.Plan(pattern, flags)
        order = p.order()
        for l in range(k):
            v = order[l]
            want = sorted([(j, 0) for j in range(l) if (order[j], v) not in aset] +
                          [(j, 1) for j in range(l) if (v, order[j]) not in aset])
            assert sorted(p.level(l)["diffs"]) == want
        assert run_plan(n, out, inn, p) == g.count_matches(pattern, induced=True)
    pe = xm.Plan(pattern, xm.XM_INDUCED | xm.XM_EMBEDDINGS)
    assert run_plan(n, out, inn, pe) == g.count_embeddings(pattern, induced=True)


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


def _weakly_connected(vertices, arcs):
    vertices = set(vertices)
    if not vertices:
        return True
    seen, todo = set(), [min(vertices)]
    while todo:
        v = todo.pop()
        if v in seen:
            continue
        seen.add(v)
        todo += [b for a, b in arcs if a == v and b in vertices] + [a for a, b in arcs if b == v and a in vertices]
    return seen == vertices


def test_product_choices():
    P = PRODUCT_PATTERNS
    expect = {"star4": (2, 2, xm.XM_PROD_CHOOSE), "star5": (2, 3, xm.XM_PROD_CHOOSE),
              "path4": (2, 2, xm.XM_PROD_IE), "ffchain5": (3, 2, xm.XM_PROD_IE),
              "mixstar": (2, 2, xm.XM_PROD_CHOOSE)}
    for name, (level, r, kind) in expect.items():
        pr = xm.Plan(P[name]).product()
        assert (pr["level"], pr["r"], pr["kind"]) == (level, r, kind), name
        assert len(pr["sets"]) == (1 if kind == xm.XM_PROD_CHOOSE else 2 ** r - 1)
    # every vertex of the 4-cycle, bi-fan and bi-parallel pattern has a
    # neighbour on each side: removing two non-adjacent ones disconnects
    for pat in (synth.CYCLE4, synth.BIFAN, synth.BIPARALLEL, synth.CYCLE3, synth.FFL):
        assert xm.Plan(pat).product()["r"] == 0
    for flags in (xm.XM_NO_PRODUCT, xm.XM_INDUCED):
        assert xm.Plan(P["star4"], flags).product()["r"] == 0
    assert "product: level 2 r=3 kind=choose" in xm.Plan(P["star5"]).describe()


@pytest.mark.parametrize("pattern", list(PRODUCT_PATTERNS.values()) + random_patterns(24, 31))
def test_product_structure(pattern):
    k, arcs = pattern
    aset = set(arcs)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE, xm.XM_EMBEDDINGS):
        p = xm.Plan(pattern, flags)
        pr = p.product()
        if pr["r"] == 0:
            assert pr["sets"] == []
            continue
        order, lvl, r = p.order(), pr["level"], pr["r"]
        assert lvl == k - r and lvl >= 2 and order[0] == p.start
        tail = order[lvl:]
        # the product vertices share no arc, the rest stays connected
        assert not any((a, b) in aset for a in tail for b in tail)
        assert _weakly_connected(order[:lvl], arcs)
        prefix = (1 << lvl) - 1
        for i, S in enumerate(pr["sets"]):
            members = [lvl + j for j in range(r) if (i + 1) >> j & 1] if pr["kind"] == xm.XM_PROD_IE else [lvl]
            want = sorted({op for m in members for op in p.level(m)["ops"]})
            assert S["vertex"] == -1 and sorted(S["ops"]) == want
            assert all(j < lvl for j, _ in S["ops"])
            assert (S["lo_mask"] | S["hi_mask"] | S["neq_mask"]) & ~prefix == 0
            assert S["dout_min"] == 0 and S["din_min"] == 0 and S["diffs"] == []
            if S["reuse"] >= 0:
                assert 1 <= S["reuse"] < lvl
                assert set(p.level(S["reuse"])["ops"]) <= set(S["ops"])
        if flags & xm.XM_EMBEDDINGS:
            assert pr["kind"] == xm.XM_PROD_IE


@pytest.mark.parametrize("seed", [5, 6])
@pytest.mark.parametrize("name", sorted(PRODUCT_PATTERNS))
def test_product_plans_vs_oracle(seed, name):
    """The product sets, counted by brute force over distinct tuples by the
    plan interpreter, give the oracle's counts."""
    pattern = PRODUCT_PATTERNS[name]
    n, src, dst = synth.er_graph(12, 60, seed=seed)
    out, inn = adjacency_lists(n, src, dst)
    g = oracle.OracleGraph(n, src, dst)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE):
        p = xm.Plan(pattern, flags)
        assert p.product()["r"] > 0
        assert run_plan(n, out, inn, p) == g.count_matches(pattern)
        assert run_plan(n, out, inn, p, use_product=False) == g.count_matches(pattern)
    pe = xm.Plan(pattern, xm.XM_EMBEDDINGS)
    assert run_plan(n, out, inn, pe) == g.count_embeddings(pattern)


# ------------------------------------------ cut-vertex decomposition (count)

SPLIT_PATTERNS = {
    "ffchain5": synth.FFCHAIN5,
    "path5": (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    "tri_tail": (5, [(0, 1), (1, 2), (0, 2), (2, 3), (2, 4)]),
    "ffl_tail": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
    "four_parts": (6, [(0, 1), (1, 0), (0, 2), (2, 3), (3, 0), (4, 0), (0, 5)]),
    "recip_path": (5, [(0, 1), (1, 0), (1, 2), (2, 3), (3, 2), (3, 4)]),
    # eight vertices: dozens of quotient classes, split again recursively
    "path8": (8, [(i, i + 1) for i in range(7)]),
    "spider8": (8, [(1, 0), (2, 1), (3, 0), (4, 3), (0, 5), (5, 6), (7, 0)]),
    "double_star8": (8, [(0, 1), (0, 2), (0, 3), (0, 4), (4, 5), (4, 6), (4, 7)]),
}


def test_split_choices():
    sp = xm.Plan(SPLIT_PATTERNS["ffchain5"]).split()
    assert sp["cut"] == 2 and len(sp["parts"]) == 2 and sp["part_factor"] == 2
    assert sorted(q["mult"] for q in sp["quotients"]) == [2, 2, 2]
    assert len(xm.Plan(SPLIT_PATTERNS["four_parts"]).split()["parts"]) == 4
    # 2-connected patterns and plans a product ends at level 2 do not split
    for pat in (synth.CYCLE4, synth.BIFAN, synth.BIPARALLEL, (4, [(0, 1), (0, 2), (0, 3)]), synth.CYCLE3):
        assert xm.Plan(pat).split()["cut"] == -1
    for flags in (xm.XM_NO_SPLIT, xm.XM_INDUCED):
        assert xm.Plan(synth.FFCHAIN5, flags).split()["cut"] == -1


SUBSET_SPLIT = dict(SPLIT_PATTERNS, **{
    # the cut vertex is the start vertex but an automorphism moves it
    "sym2": (6, [(0, 1), (1, 0), (0, 2), (2, 3), (1, 4), (4, 5)]),
    "twotri": (6, [(0, 1), (1, 0), (0, 2), (2, 3), (3, 0), (1, 4), (4, 5), (5, 1)]),
    "sym3": (7, [(0, 1), (1, 0), (0, 2), (2, 3), (3, 0), (1, 4), (4, 5), (5, 1), (6, 0)]),
})


@pytest.mark.parametrize("name", sorted(SUBSET_SPLIT))
def test_split_over_start_node_subsets_choice(name):
    """Counts over a start-node range or list use the decomposition exactly
    when the cut vertex is the plan's start vertex and every automorphism
    (the oracle's, by brute force) fixes it: then all embeddings of a match
    send the cut vertex to one node, and per-node sums are exact."""
    pattern = SUBSET_SPLIT[name]
    plan = xm.Plan(pattern)
    sp = plan.split()
    if sp["cut"] < 0:
        return
    fixed = all(row[sp["cut"]] == sp["cut"] for row in oracle.automorphisms(pattern))
    want = "split" if (sp["cut"] == plan.start and fixed) else "walked"
    line = [ln for ln in plan.describe().splitlines() if ln.startswith("cut-vertex split:")]
    assert line and line[0].endswith("start-node subsets " + want), (name, line)
    for name2, w in (("ffchain5", "split"), ("bowtie", "split"), ("sym2", "walked"), ("path5", "walked")):
        if name == name2:
            assert want == w


@pytest.mark.parametrize("seed", [7, 8])
@pytest.mark.parametrize("name", sorted(SPLIT_PATTERNS))
def test_split_identity_vs_oracle(seed, name):
    """The decomposition's parts, stabilisers, quotients and multiplicities,
    evaluated with the oracle alone: sum over nodes v of the product of the
    parts' embeddings rooted at v, minus the quotients' embeddings, is the
    pattern's embedding count."""
    pattern = SPLIT_PATTERNS[name]
    k, arcs = pattern
    n, src, dst = synth.er_graph(11, 70, seed=seed)
    g = oracle.OracleGraph(n, src, dst)
    for flags in (xm.XM_REDUCE, xm.XM_NO_REDUCE, xm.XM_EMBEDDINGS, xm.XM_NO_PRODUCT):
        plan = xm.Plan(pattern, flags)
        sp = plan.split()
        if sp["cut"] < 0:
            # a leaf product that stops the walk at level 2 is kept instead
            assert plan.product()["level"] == 2 and not flags & xm.XM_NO_PRODUCT, name
            continue
        cut = sp["cut"]
        seen = set()
        factor = 1
        for part in sp["parts"]:
            pk, parcs = part["pattern"]
            vs = part["vertices"]
            assert vs[0] == cut and len(vs) == pk
            assert not (set(vs[1:]) & seen)
            seen |= set(vs[1:])
            # the part is the induced sub-pattern on its vertices, relabelled
            assert sorted((vs[a], vs[b]) for a, b in parcs) == \
                sorted((a, b) for a, b in arcs if a in vs and b in vs)
            aut = oracle.automorphisms(part["pattern"])
            assert part["stab"] == sum(1 for row in aut if row[0] == 0)
            factor *= part["stab"]
        assert seen == set(range(k)) - {cut} and sp["part_factor"] == factor
        total = 0
        for v in range(n):
            prod = 1
            for part in sp["parts"]:
                prod *= g.count_embeddings(part["pattern"], 0, v, v + 1)
            total += prod
        for q in sp["quotients"]:
            assert q["pattern"][0] < k and q["mult"] >= 1
            total -= q["mult"] * g.count_embeddings(q["pattern"])
        assert total == g.count_embeddings(pattern)
        if "start-node subsets split" in plan.describe():
            # node by node: the embeddings mapping the cut vertex to v are the
            # parts' products at v minus the quotients' embeddings rooted at v
            # (the cut vertex is label 0 of every quotient)
            assert plan.start == cut
            for v in range(n):
                per = 1
                for part in sp["parts"]:
                    per *= g.count_embeddings(part["pattern"], 0, v, v + 1)
                for q in sp["quotients"]:
                    per -= q["mult"] * g.count_embeddings(q["pattern"], 0, v, v + 1)
                assert per == g.count_embeddings(pattern, cut, v, v + 1), (name, v)
