"""Failure handling without faulting a GPU.

* Host-side: bad arguments come back as status codes (no exceptions across
  the ABI, no crash).
* Device-side: a matcher whose work budget runs out stops at its next check,
  returns XM_ETIMEOUT with no count, and the context stays usable -- the
  next call returns the exact count. Nothing here traps, hangs or makes an
  invalid access.
"""
import ctypes

import numpy as np
import pytest

import synth
import paper_2404_11105_b300 as xm


def test_null_arguments_return_einval():
    L = xm.lib()
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    assert L.xm_count(None, None, ctypes.byref(lo), ctypes.byref(hi), None) == xm.XM_EINVAL
    assert b"NULL" in L.xm_last_error()
    assert L.xm_compile_pattern(3, 2, None, None, 0, ctypes.byref(ctypes.c_void_p())) == xm.XM_EINVAL
    assert L.xm_plan_info(None, None, None, None, None, None) == xm.XM_EINVAL
    assert L.xm_batch_run(None, None) == xm.XM_EINVAL
    assert L.xm_strerror(99) == b"XM_UNKNOWN"


def test_product_and_split_queries_reject_bad_arguments():
    L = xm.lib()
    info = xm.xm_level_info()
    i32 = ctypes.c_int32
    assert L.xm_plan_product(None, None, None, None, None) == xm.XM_EINVAL
    assert L.xm_plan_split(None, None, None, None, None) == xm.XM_EINVAL
    star = xm.Plan((4, [(0, 1), (0, 2), (0, 3)]))           # choose product, no split
    assert L.xm_plan_product_set(star._h, 1, ctypes.byref(info)) == xm.XM_EINVAL
    assert L.xm_plan_product_set(star._h, -1, ctypes.byref(info)) == xm.XM_EINVAL
    assert L.xm_plan_product_set(star._h, 0, ctypes.byref(info)) == xm.XM_OK
    buf = (i32 * 56)()
    assert L.xm_plan_split_part(star._h, 0, None, None, buf, buf, None, None) == xm.XM_EINVAL
    assert L.xm_plan_split_quotient(star._h, 0, None, None, buf, buf, None) == xm.XM_EINVAL
    chain = xm.Plan(synth.FFCHAIN5)
    sp = chain.split()
    assert L.xm_plan_split_part(chain._h, len(sp["parts"]), None, None, buf, buf, None, None) == xm.XM_EINVAL
    assert L.xm_plan_split_quotient(chain._h, len(sp["quotients"]), None, None, buf, buf, None) == xm.XM_EINVAL
    # unknown flag bits
    ps, pd = (i32 * 1)(0), (i32 * 1)(1)
    assert L.xm_compile_pattern(2, 1, ps, pd, 32, ctypes.byref(ctypes.c_void_p())) == xm.XM_EINVAL


def test_bad_tuning_rejected():
    p = xm.Plan(synth.FFL)
    for bad in (dict(window=48), dict(unit=0, window=5000), dict(warps_per_block=17), dict(budget_ms=-1)):
        with pytest.raises(xm.XmError) as ei:
            p.set_tuning(**bad)
        assert ei.value.status == xm.XM_EINVAL
    assert p.tuning()["window"] == 512  # unchanged


@pytest.mark.gpu
def test_time_budget_gives_etimeout_and_context_survives():
    n, src, dst = synth.rmat_graph(18, 16, seed=8)
    g = xm.Graph(n, src, dst)
    p = xm.Plan(synth.FFL)
    want = xm.xm_count(g, p)
    p.set_tuning(budget_ms=1)
    hit = False
    for _ in range(3):  # a 1 ms budget on a multi-ms count
        try:
            xm.xm_count(g, p)
        except xm.XmError as e:
            assert e.status == xm.XM_ETIMEOUT
            hit = True
            break
    assert hit
    p.set_tuning(budget_ms=0)
    assert xm.xm_count(g, p) == want
    # the batched kernel honours its budget the same way
    b = xm.Batch([p], [g], [(0, 0)])
    b.set_tuning(budget_ms=1)
    b.run()
    with pytest.raises(xm.XmError) as ei:
        b.counts()
    assert ei.value.status == xm.XM_ETIMEOUT
    b.set_tuning(budget_ms=0)
    b.run()
    assert b.counts() == [want]
