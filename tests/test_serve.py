"""Serving: queries admitted into slots by scratch memory, overlapping on
the GPU. Each query's count is the same alone (xm_count) and in the mix;
admission never exceeds the memory budget; a query over its time budget
completes with XM_ETIMEOUT without disturbing the others."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xm():
    import paper_2404_11105_b300 as m
    return m


@pytest.fixture(scope="module")
def world(xm):
    graphs = [xm.Graph(*synth.small_graph(i, seed=61, n_lo=50, n_hi=800)) for i in range(12)]
    graphs.append(xm.Graph(*synth.rmat_graph(14, 8, seed=62)))
    pats = [synth.CYCLE3, synth.FFL, synth.BIFAN, synth.CYCLE4, synth.FFCHAIN5] + \
           [synth.batch_pattern(i, seed=63, k_hi=4) for i in range(5)]
    plans = [xm.Plan(p) for p in pats]
    queries = [(qi % len(plans), (qi * 7) % len(graphs)) for qi in range(60)]
    alone = [xm.xm_count(graphs[gi], plans[pi]) for pi, gi in queries]
    return graphs, plans, queries, alone


def drain(srv, queries, plans, results, max_busy=None):
    pending = list(range(len(queries)))
    while pending or srv.info()[0]:
        progressed = False
        while pending:
            q = pending[0]
            pi, gi = queries[q]
            if not srv.submit(plans[pi], gi, q):
                break
            pending.pop(0)
            progressed = True
            if max_busy is not None:
                assert srv.info()[0] <= max_busy
        for tag, c, st in srv.poll(wait=not progressed):
            results[tag] = (c, st)


def test_results_same_alone_and_in_the_mix(xm, world):
    graphs, plans, queries, alone = world
    srv = xm.Server(graphs, slots=6)
    results = {}
    drain(srv, queries, plans, results)
    assert len(results) == len(queries)
    for q, want in enumerate(alone):
        assert results[q] == (want, xm.XM_OK), q
    srv.free()


def test_admission_respects_memory_budget(xm, world):
    graphs, plans, queries, alone = world
    big = max(xm.xm_query_bytes(g, plans[0]) for g in graphs)
    # room for one largest query at a time (plus nothing else)
    srv = xm.Server(graphs, slots=6, mem_budget_bytes=big)
    results = {}
    pending = list(range(len(queries)))
    while pending or srv.info()[0]:
        while pending:
            pi, gi = queries[pending[0]]
            if not srv.submit(plans[pi], gi, pending[0]):
                break
            pending.pop(0)
            assert srv.info()[1] <= big
        for tag, c, st in srv.poll(wait=True):
            results[tag] = (c, st)
    assert [results[q][0] for q in range(len(queries))] == alone
    srv.free()
    with pytest.raises(xm.XmError):
        tiny = xm.Server(graphs, slots=2, mem_budget_bytes=1024)
        tiny.submit(plans[0], 0, 0)


def test_timeout_in_the_mix(xm, world):
    graphs, plans, queries, alone = world
    heavy = xm.Graph(*synth.rmat_graph(18, 16, seed=8))
    slow = xm.Plan(synth.FFL)
    slow.set_tuning(budget_ms=1)
    srv = xm.Server(graphs + [heavy], slots=4)
    assert srv.submit(slow, len(graphs), 999)
    results = {}
    drain(srv, queries[:10], plans, results)
    while srv.info()[0]:
        for tag, c, st in srv.poll(wait=True):
            results[tag] = (c, st)
    for tag, c, st in srv.poll():
        results[tag] = (c, st)
    assert results[999] == (None, xm.XM_ETIMEOUT)
    for q in range(10):
        assert results[q] == (alone[q], xm.XM_OK)
    srv.free()
