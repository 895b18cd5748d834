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


# ------------------------------------------------ host-side fault injection

def test_injected_compile_fault_and_spec_parsing():
    """compile:N makes exactly the N-th compile from now fail (XM_ENOMEM),
    the ones before and after succeed; malformed specs are refused."""
    try:
        xm.fault_inject("compile:2")
        xm.Plan(synth.FFL)
        with pytest.raises(xm.XmError) as ei:
            xm.Plan(synth.BIFAN)
        assert ei.value.status == xm.XM_ENOMEM and "injected" in str(ei.value)
        xm.Plan(synth.BIFAN)
        for bad in ("alloc:0", "alloc", "alloc:x", "disk:1", "compile:-3", ""):
            with pytest.raises(xm.XmError) as ei:
                xm.fault_inject(bad)
            assert ei.value.status == xm.XM_EINVAL
        xm.fault_inject("compile:1,none")
        xm.Plan(synth.FFL)
    finally:
        xm.fault_inject("none")


def test_xm_fault_environment_variable():
    """XM_FAULT is read when the library loads (a fresh process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); import synth, paper_2404_11105_b300 as xm\n"
            "xm.Plan(synth.FFL)\n"
            "try:\n    xm.Plan(synth.FFL)\n    print('no fault')\n"
            "except xm.XmError as e:\n    print('fault', e.status)\n" % root)
    out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, XM_FAULT="compile:2"),
                         capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "fault %d" % xm.XM_ENOMEM, out.stderr


@pytest.mark.gpu
def test_injected_allocation_faults_leak_nothing():
    """Every device allocation of a graph load, a per-root count, a batch
    and a server in turn made to fail: each call reports XM_ENOMEM, the
    library holds exactly the bytes it held before, and the same call then
    succeeds with the right count."""
    n, src, dst = synth.er_graph(400, 3000, seed=7)
    base = xm.device_bytes_live()
    want = xm.xm_count(xm.Graph(n, src, dst), xm.Plan(synth.BIFAN))
    assert xm.device_bytes_live() == base
    try:
        nth = 1
        while True:
            xm.fault_inject(f"alloc:{nth}")
            try:
                g = xm.Graph(n, src, dst)
            except xm.XmError as e:
                assert e.status == xm.XM_ENOMEM
                assert xm.device_bytes_live() == base, nth
                nth += 1
                continue
            xm.fault_inject("none")
            break
        assert nth > 10  # every allocation of the load was hit once
        assert xm.xm_count(g, xm.Plan(synth.BIFAN)) == want
        # per-root counters and the root buffer, allocated on first use
        held = xm.device_bytes_live()
        p = xm.Plan(synth.BIFAN)
        for spec in ("alloc:1", "alloc:2"):
            xm.fault_inject(spec)
            with pytest.raises(xm.XmError) as ei:
                xm.xm_count_roots_each(g, p, np.arange(50, dtype=np.int32))
            assert ei.value.status == xm.XM_ENOMEM
        xm.fault_inject("none")
        assert sum(xm.xm_count_roots_each(g, p, np.arange(n, dtype=np.int32))) == want
        assert xm.device_bytes_live() >= held
        # a batch
        held = xm.device_bytes_live()
        for nth in range(1, 7):
            xm.fault_inject(f"alloc:{nth}")
            with pytest.raises(xm.XmError) as ei:
                xm.Batch([p], [g], [(0, 0)])
            assert ei.value.status == xm.XM_ENOMEM
            assert xm.device_bytes_live() == held
        xm.fault_inject("none")
        assert xm.xm_count_batch([p], [g], [(0, 0)]) == [want]
        # a query whose scratch cannot be allocated is not admitted (the
        # caller retries), and nothing is held for it
        srv = xm.Server([g], slots=2, mem_budget_bytes=1 << 30)
        held = xm.device_bytes_live()
        xm.fault_inject("alloc:1")
        assert not srv.submit(p, 0, 7)
        xm.fault_inject("none")
        assert xm.device_bytes_live() == held and srv.info()[0] == 0
        assert srv.submit(p, 0, 8)
        res = srv.poll(wait=True)
        assert [(t, c, s) for t, c, s in res] == [(8, want, xm.XM_OK)]
        srv.free()
        g.free()
        assert xm.device_bytes_live() == base
    finally:
        xm.fault_inject("none")
