"""The allocation-free count entry point (xm_count_noalloc) against xm_count.

Callers that cannot allocate device memory (a process whose device memory
is all handed to its own pool up front, or a loop that must not pay for
cudaMalloc/cudaFree) use xm_count_noalloc with their own CSR arrays; the
library then works in its fixed, file-scope scratch area. This file is
collected last so that a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xm():
    import paper_2404_11105_b300 as m
    return m


def _noalloc(xm, g, p):
    oo, oa, io, ia = g.csr_pointers()
    return xm.xm_count_noalloc(oo, oa, io, ia, g.n, g.m, p)


@pytest.mark.parametrize("graph", ["tiny_er", "rmat12"])
def test_noalloc_matches_xm_count_twice(xm, graph):
    if graph == "tiny_er":
        n, src, dst = synth.tiny_er()
    else:
        n, src, dst = synth.rmat_graph(12, 8, seed=31)
    g = xm.Graph(n, src, dst)
    pats = [synth.CYCLE3, synth.FFL, synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5, (2, [(0, 1)])]
    for pat in pats:
        p = xm.Plan(pat)
        want = xm.xm_count(g, p)
        # two calls in a row: the shared scratch keeps the previous contents
        assert _noalloc(xm, g, p) == want
        assert _noalloc(xm, g, p) == want
    # a different graph between calls on the same scratch
    n2, s2, d2 = synth.er_graph(300, 2500, seed=4)
    g2 = xm.Graph(n2, s2, d2)
    p = xm.Plan(synth.BIFAN)
    assert _noalloc(xm, g2, p) == xm.xm_count(g2, p)
    assert _noalloc(xm, g, p) == xm.xm_count(g, p)


def test_noalloc_rejects_graphs_beyond_its_scratch(xm):
    n, src, dst = synth.rmat_graph(21, 2, seed=5)   # needs more than the 32 MiB area
    g = xm.Graph(n, src, dst)
    with pytest.raises(xm.XmError) as ei:
        _noalloc(xm, g, xm.Plan(synth.FFL))
    assert ei.value.status == xm.XM_EINVAL
    assert "too large" in str(ei.value)


def test_noalloc_near_its_limit_with_hub_lists(xm):
    """A skewed graph whose scratch nearly fills the fixed area: hub lists of
    hundreds of ids take the paths that differ between the two entry points
    (xm_count probes hash tables and counts three-vertex levels from
    registers; the allocation-free call has no hash tables and falls back to
    merges and binary searches)."""
    n, src, dst = synth.rmat_graph(17, 16, seed=41)
    g = xm.Graph(n, src, dst)
    need = 4 * (3 * g.n + 3.001 * g.m)
    assert 0.6 * (32 << 20) < need < (32 << 20)
    oo, oa, io, ia = g.csr_pointers()
    for pat in (synth.CYCLE3, synth.FFL, synth.MOTIFS3["030T"], synth.BIPARALLEL,
                (4, [(0, 1), (1, 2), (2, 3)])):
        p = xm.Plan(pat)
        want = xm.xm_count(g, p)
        assert want > 0
        assert xm.xm_count_noalloc(oo, oa, io, ia, g.n, g.m, p) == want
        assert xm.xm_count_noalloc(oo, oa, io, ia, g.n, g.m, p) == want


def test_noalloc_rejects_inconsistent_arc_counts(xm):
    """m must equal out_off[n] and in_off[n]: a wrong m is refused before
    any kernel runs, and the next correct call still works."""
    n, src, dst = synth.er_graph(300, 2500, seed=4)
    g = xm.Graph(n, src, dst)
    oo, oa, io, ia = g.csr_pointers()
    p = xm.Plan(synth.BIFAN)
    for bad_m in (g.m + 1, g.m - 1, 0):
        with pytest.raises(xm.XmError) as ei:
            xm.xm_count_noalloc(oo, oa, io, ia, g.n, bad_m, p)
        assert ei.value.status == xm.XM_EINVAL
    assert xm.xm_count_noalloc(oo, oa, io, ia, g.n, g.m, p) == xm.xm_count(g, p)
