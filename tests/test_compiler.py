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
    assert p.tuning() == {"window": 256, "unit": 16, "warps_per_block": 4, "blocks_per_sm": 2, "budget_ms": 0}
    with pytest.raises(xm.XmError):
        p.set_tuning(window=100)


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
