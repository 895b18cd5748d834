"""Python binding of the B300 directed subgraph matcher (libxm.so).

Argument marshalling only: every step of matching runs in the CUDA library
behind the C ABI of include/xm.h (graph build and pattern compilation run
in its host C++ code). PyTorch supplies device memory and streams.

The library must have been built in-tree (``python -m
paper_2404_11105_b300.build``); the first call into this package raises
when it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxm.so")

XM_OK, XM_EINVAL, XM_ENOMEM, XM_EOVERFLOW, XM_ECUDA, XM_ETIMEOUT, XM_EBUSY = range(7)
XM_REDUCE, XM_NO_REDUCE, XM_EMBEDDINGS, XM_INDUCED, XM_NO_PRODUCT, XM_NO_SPLIT = 0, 1, 2, 4, 8, 16
XM_PROD_NONE, XM_PROD_CHOOSE, XM_PROD_IE = 0, 1, 2

# every symbol include/xm.h declares
EXPORTS = ["xm_strerror", "xm_last_error", "xm_version", "xm_load_graph", "xm_graph_info", "xm_graph_csr",
           "xm_graph_free", "xm_compile_pattern", "xm_plan_info", "xm_plan_order", "xm_plan_level",
           "xm_plan_describe", "xm_plan_free", "xm_plan_set_tuning", "xm_plan_get_tuning", "xm_count",
           "xm_count_range", "xm_count_stats", "xm_enumerate", "xm_enumerate_range", "xm_graph_last_timing",
           "xm_count_noalloc", "xm_batch_create", "xm_batch_set_tuning", "xm_batch_get_tuning", "xm_batch_run",
           "xm_batch_run_graph", "xm_batch_counts", "xm_batch_tune", "xm_batch_free", "xm_count_batch",
           "xm_query_bytes", "xm_server_create", "xm_server_submit", "xm_server_poll", "xm_server_info",
           "xm_server_free", "xm_count_roots", "xm_enumerate_roots", "xm_count_roots_stats", "xm_plan_tune",
           "xm_plan_product", "xm_plan_product_set", "xm_plan_split", "xm_plan_split_part",
           "xm_plan_split_quotient", "xm_count_roots_each", "xm_plan_tune_roots", "xm_fault_inject",
           "xm_device_bytes_live", "xm_batch_set_pair_budget", "xm_batch_pair_status"]


class XmError(RuntimeError):
    def __init__(self, status: int, detail: str):
        self.status = status
        super().__init__(f"{lib().xm_strerror(status).decode()}: {detail}")


class xm_tuning(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("unit", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("budget_ms", ctypes.c_int32), ("merge_ratio", ctypes.c_int32)]


class xm_stats(ctypes.Structure):
    _fields_ = [("alg_bytes", ctypes.c_uint64), ("extensions", ctypes.c_uint64), ("set_ops", ctypes.c_uint64),
                ("units", ctypes.c_uint64), ("leaf_elems", ctypes.c_uint64), ("l1_bytes", ctypes.c_uint64),
                ("touched_bytes", ctypes.c_uint64), ("warp_exit_first_ns", ctypes.c_uint64),
                ("warp_exit_mean_ns", ctypes.c_uint64), ("warp_exit_last_ns", ctypes.c_uint64)]


class xm_level_info(ctypes.Structure):
    _fields_ = [("vertex", ctypes.c_int32), ("nops", ctypes.c_int32), ("op_level", ctypes.c_int32 * 14),
                ("op_dir", ctypes.c_int32 * 14), ("reuse", ctypes.c_int32), ("reuse_ops", ctypes.c_uint32),
                ("dout_min", ctypes.c_int32), ("din_min", ctypes.c_int32), ("lo_mask", ctypes.c_uint32),
                ("hi_mask", ctypes.c_uint32), ("neq_mask", ctypes.c_uint32), ("ndiff", ctypes.c_int32),
                ("diff_level", ctypes.c_int32 * 14), ("diff_dir", ctypes.c_int32 * 14)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_11105_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "xm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "xm_last_error": (ctypes.c_char_p, []),
        "xm_version": (ctypes.c_int, []),
        "xm_fault_inject": (ctypes.c_int, [ctypes.c_char_p]),
        "xm_device_bytes_live": (ctypes.c_uint64, []),
        "xm_load_graph": (ctypes.c_int, [i32, i64, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "xm_graph_info": (ctypes.c_int, [vp, i32p, ctypes.POINTER(i64)]),
        "xm_graph_csr": (ctypes.c_int, [vp] + [ctypes.POINTER(vp)] * 4),
        "xm_graph_free": (None, [vp]),
        "xm_compile_pattern": (ctypes.c_int, [i32, i32, i32p, i32p, ctypes.c_int, ctypes.POINTER(vp)]),
        "xm_plan_info": (ctypes.c_int, [vp, i32p, i32p, i32p, i32p, i32p]),
        "xm_plan_order": (ctypes.c_int, [vp, i32p]),
        "xm_plan_level": (ctypes.c_int, [vp, i32, ctypes.POINTER(xm_level_info)]),
        "xm_plan_product": (ctypes.c_int, [vp, i32p, i32p, i32p, i32p]),
        "xm_plan_product_set": (ctypes.c_int, [vp, i32, ctypes.POINTER(xm_level_info)]),
        "xm_plan_split": (ctypes.c_int, [vp, i32p, i32p, i32p, ctypes.POINTER(i64)]),
        "xm_plan_split_part": (ctypes.c_int, [vp, i32, i32p, i32p, i32p, i32p, i32p, i32p]),
        "xm_plan_split_quotient": (ctypes.c_int, [vp, i32, i32p, i32p, i32p, i32p, ctypes.POINTER(i64)]),
        "xm_plan_describe": (ctypes.c_int, [vp, ctypes.c_char_p, i32]),
        "xm_plan_free": (None, [vp]),
        "xm_plan_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(xm_tuning)]),
        "xm_plan_get_tuning": (ctypes.c_int, [vp, ctypes.POINTER(xm_tuning)]),
        "xm_count": (ctypes.c_int, [vp, vp, u64p, u64p, vp]),
        "xm_count_range": (ctypes.c_int, [vp, vp, i64, i64, u64p, u64p, vp]),
        "xm_count_stats": (ctypes.c_int, [vp, vp, i64, i64, u64p, u64p, ctypes.POINTER(xm_stats), vp]),
        "xm_enumerate": (ctypes.c_int, [vp, vp, vp, ctypes.c_uint64, u64p, u64p, vp]),
        "xm_enumerate_range": (ctypes.c_int, [vp, vp, i64, i64, vp, ctypes.c_uint64, u64p, u64p, vp]),
        "xm_graph_last_timing": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "xm_count_noalloc": (ctypes.c_int, [vp, vp, vp, vp, i32, i64, vp, u64p, u64p, vp]),
        "xm_batch_create": (ctypes.c_int, [i32, ctypes.POINTER(vp), i32, ctypes.POINTER(vp), i64, i32p,
                                           ctypes.POINTER(vp)]),
        "xm_batch_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(xm_tuning)]),
        "xm_batch_get_tuning": (ctypes.c_int, [vp, ctypes.POINTER(xm_tuning)]),
        "xm_batch_run": (ctypes.c_int, [vp, vp]),
        "xm_batch_run_graph": (ctypes.c_int, [vp, vp]),
        "xm_batch_counts": (ctypes.c_int, [vp, u64p, vp]),
        "xm_batch_tune": (ctypes.c_int, [vp, ctypes.POINTER(xm_tuning), i32, i32, ctypes.POINTER(xm_tuning),
                                         ctypes.POINTER(ctypes.c_float), vp]),
        "xm_batch_free": (None, [vp]),
        "xm_batch_set_pair_budget": (ctypes.c_int, [vp, i32]),
        "xm_batch_pair_status": (ctypes.c_int, [vp, i32p, vp]),
        "xm_count_batch": (ctypes.c_int, [i32, ctypes.POINTER(vp), i32, ctypes.POINTER(vp), i64, i32p, u64p, vp]),
        "xm_query_bytes": (ctypes.c_uint64, [vp, vp]),
        "xm_count_roots": (ctypes.c_int, [vp, vp, i32p, i64, u64p, u64p, vp]),
        "xm_count_roots_each": (ctypes.c_int, [vp, vp, i32p, i64, u64p, vp]),
        "xm_plan_tune": (ctypes.c_int, [vp, vp, ctypes.POINTER(xm_tuning), i32, i32, ctypes.POINTER(xm_tuning),
                                        ctypes.POINTER(ctypes.c_float), vp]),
        "xm_count_roots_stats": (ctypes.c_int, [vp, vp, i32p, i64, u64p, u64p, ctypes.POINTER(xm_stats), vp]),
        "xm_plan_tune_roots": (ctypes.c_int, [vp, vp, i32p, i64, ctypes.POINTER(xm_tuning), i32, i32,
                                              ctypes.POINTER(xm_tuning), ctypes.POINTER(ctypes.c_float), vp]),
        "xm_enumerate_roots": (ctypes.c_int, [vp, vp, i32p, i64, vp, ctypes.c_uint64, u64p, u64p, vp]),
        "xm_server_create": (ctypes.c_int, [i32, ctypes.POINTER(vp), i32, ctypes.c_uint64, ctypes.POINTER(vp)]),
        "xm_server_submit": (ctypes.c_int, [vp, vp, i32, i64, i32p]),
        "xm_server_poll": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(ctypes.c_int64), u64p, i32p, i32p]),
        "xm_server_info": (ctypes.c_int, [vp, i32p, u64p]),
        "xm_server_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    """The loaded libxm.so (ctypes); raises if it has not been built."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def _check(rc: int):
    if rc != XM_OK:
        raise XmError(rc, lib().xm_last_error().decode())


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _ptr(x):
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.int32 and x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    assert str(x.dtype) == "torch.int32" and x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


class Graph:
    """Data digraph resident on the current CUDA device (dual sorted CSR)."""

    def __init__(self, n: int, src, dst, stream=None):
        h = ctypes.c_void_p()
        self._keep = (src, dst)
        _check(lib().xm_load_graph(int(n), len(src), _ptr(src), _ptr(dst), 0, _stream(stream), ctypes.byref(h)))
        self._keep = None
        self._h = h
        n_ = ctypes.c_int32()
        m_ = ctypes.c_int64()
        _check(lib().xm_graph_info(h, ctypes.byref(n_), ctypes.byref(m_)))
        self.n, self.m = n_.value, m_.value

    def csr_pointers(self):
        ps = [ctypes.c_void_p() for _ in range(4)]
        _check(lib().xm_graph_csr(self._h, *[ctypes.byref(p) for p in ps]))
        return [p.value for p in ps]

    def csr_host(self):
        """Copies of the device CSR as numpy int32 arrays (out_off, out_adj,
        in_off, in_adj); torch moves the bytes."""
        import torch

        class _View:  # a device array by pointer, for torch.as_tensor
            def __init__(self, ptr, count):
                self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<i4", "data": (ptr, False),
                                                 "version": 3}

        oo, oa, io, ia = self.csr_pointers()
        sizes = (self.n + 1, self.m, self.n + 1, self.m)
        return [torch.as_tensor(_View(p, c), device="cuda").cpu().numpy() if c else np.zeros(0, np.int32)
                for p, c in zip((oo, oa, io, ia), sizes)]

    def last_timing(self):
        """(prep_ms, match_ms) of the last call, from CUDA events on its stream."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(lib().xm_graph_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free(self):
        if getattr(self, "_h", None):
            lib().xm_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """Compiled pattern (host-only)."""

    def __init__(self, pattern, flags: int = XM_REDUCE):
        k, arcs = pattern
        ps = (ctypes.c_int32 * len(arcs))(*[a for a, _ in arcs])
        pd = (ctypes.c_int32 * len(arcs))(*[b for _, b in arcs])
        h = ctypes.c_void_p()
        _check(lib().xm_compile_pattern(k, len(arcs), ps, pd, flags, ctypes.byref(h)))
        self._h = h
        self.pattern = (k, list(arcs))
        self.flags = flags
        vals = [ctypes.c_int32() for _ in range(5)]
        _check(lib().xm_plan_info(h, *[ctypes.byref(v) for v in vals]))
        self.k, self.aut_size, self.n_levels, self.n_reuse, self.start = [v.value for v in vals]

    def order(self):
        o = (ctypes.c_int32 * self.k)()
        _check(lib().xm_plan_order(self._h, o))
        return list(o)

    @staticmethod
    def _level_dict(info) -> dict:
        return {"vertex": info.vertex, "ops": [(info.op_level[i], info.op_dir[i]) for i in range(info.nops)],
                "reuse": info.reuse, "reuse_ops": info.reuse_ops, "dout_min": info.dout_min,
                "din_min": info.din_min, "lo_mask": info.lo_mask, "hi_mask": info.hi_mask,
                "neq_mask": info.neq_mask,
                "diffs": [(info.diff_level[i], info.diff_dir[i]) for i in range(info.ndiff)]}

    def level(self, l: int) -> dict:
        info = xm_level_info()
        _check(lib().xm_plan_level(self._h, l, ctypes.byref(info)))
        return self._level_dict(info)

    def product(self) -> dict:
        """Leaf product of the plan: level p, r vertices, kind, and its sets."""
        vals = [ctypes.c_int32() for _ in range(4)]
        _check(lib().xm_plan_product(self._h, *[ctypes.byref(v) for v in vals]))
        level, r, kind, n = [v.value for v in vals]
        sets = []
        for i in range(n):
            info = xm_level_info()
            _check(lib().xm_plan_product_set(self._h, i, ctypes.byref(info)))
            sets.append(self._level_dict(info))
        return {"level": level, "r": r, "kind": kind, "sets": sets}

    def split(self) -> dict:
        """Cut-vertex decomposition used by xm_count: the cut vertex (-1:
        none), the parts as rooted patterns (root 0) with their vertices in
        the original pattern and stabiliser sizes, and the quotient patterns
        with multiplicities."""
        cut, npart, nquot = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        factor = ctypes.c_int64()
        _check(lib().xm_plan_split(self._h, ctypes.byref(cut), ctypes.byref(npart), ctypes.byref(nquot),
                                   ctypes.byref(factor)))
        parts, quots = [], []
        for i in range(npart.value):
            k, e, stab = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            ps, pd, vs = (ctypes.c_int32 * 56)(), (ctypes.c_int32 * 56)(), (ctypes.c_int32 * 8)()
            _check(lib().xm_plan_split_part(self._h, i, ctypes.byref(k), ctypes.byref(e), ps, pd, vs,
                                            ctypes.byref(stab)))
            parts.append({"pattern": (k.value, [(ps[a], pd[a]) for a in range(e.value)]),
                          "vertices": list(vs[: k.value]), "stab": stab.value})
        for i in range(nquot.value):
            k, e, mult = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
            ps, pd = (ctypes.c_int32 * 56)(), (ctypes.c_int32 * 56)()
            _check(lib().xm_plan_split_quotient(self._h, i, ctypes.byref(k), ctypes.byref(e), ps, pd,
                                                ctypes.byref(mult)))
            quots.append({"pattern": (k.value, [(ps[a], pd[a]) for a in range(e.value)]), "mult": mult.value})
        return {"cut": cut.value, "parts": parts, "part_factor": factor.value, "quotients": quots}

    def describe(self) -> str:
        need = lib().xm_plan_describe(self._h, None, 0)
        buf = ctypes.create_string_buffer(need + 1)
        lib().xm_plan_describe(self._h, buf, need + 1)
        return buf.value.decode()

    def set_tuning(self, window=0, unit=0, warps_per_block=0, blocks_per_sm=0, budget_ms=0, merge_ratio=0):
        t = xm_tuning(window, unit, warps_per_block, blocks_per_sm, budget_ms, merge_ratio)
        _check(lib().xm_plan_set_tuning(self._h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = xm_tuning()
        _check(lib().xm_plan_get_tuning(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in xm_tuning._fields_}

    def free(self):
        if getattr(self, "_h", None):
            lib().xm_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fault_inject(spec: str):
    """Host-side fault injection ("alloc:N", "compile:N", "none")."""
    _check(lib().xm_fault_inject(spec.encode()))


def device_bytes_live() -> int:
    """Device bytes the library currently holds."""
    return int(lib().xm_device_bytes_live())


def xm_count(g: Graph, p: Plan, stream=None) -> int:
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().xm_count(g._h, p._h, ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return (hi.value << 64) | lo.value


def xm_count_range(g: Graph, p: Plan, root_lo: int, root_hi: int, stream=None) -> int:
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().xm_count_range(g._h, p._h, root_lo, root_hi, ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return (hi.value << 64) | lo.value


def xm_count_stats(g: Graph, p: Plan, root_lo: int = 0, root_hi: int | None = None, stream=None):
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    st = xm_stats()
    root_hi = g.n if root_hi is None else root_hi
    _check(lib().xm_count_stats(g._h, p._h, root_lo, root_hi, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(st),
                               _stream(stream)))
    return (hi.value << 64) | lo.value, {f: getattr(st, f) for f, _ in xm_stats._fields_ if f != "reserved"}


def xm_enumerate(g: Graph, p: Plan, out, capacity: int | None = None, root_lo: int = 0, root_hi: int | None = None,
                 stream=None):
    """Writes matches into the int32 device tensor `out` (capacity * k
    entries). Returns (total, written); total is exact even on overflow."""
    cap = out.numel() // p.k if capacity is None else capacity
    assert out.numel() >= cap * p.k
    total, written = ctypes.c_uint64(), ctypes.c_uint64()
    root_hi = g.n if root_hi is None else root_hi
    rc = lib().xm_enumerate_range(g._h, p._h, root_lo, root_hi, _ptr(out), cap, ctypes.byref(total),
                                 ctypes.byref(written), _stream(stream))
    if rc not in (XM_OK, XM_EOVERFLOW):
        _check(rc)
    return total.value, written.value, rc == XM_EOVERFLOW


def xm_count_noalloc(out_off, out_adj, in_off, in_adj, n: int, m: int, p: Plan, stream=None) -> int:
    """Count on caller-owned device CSR arrays (raw device pointers as ints)
    without any device allocation: the library's fixed scratch area is used
    (see include/xm.h for the size limit and the concurrency rule)."""
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().xm_count_noalloc(ctypes.c_void_p(out_off), ctypes.c_void_p(out_adj), ctypes.c_void_p(in_off),
                                  ctypes.c_void_p(in_adj), n, m, p._h, ctypes.byref(lo), ctypes.byref(hi),
                                  _stream(stream)))
    return (hi.value << 64) | lo.value


class Batch:
    """Many (plan, graph) pairs matched in one persistent launch."""

    def __init__(self, plans, graphs, pairs):
        self._plans, self._graphs = list(plans), list(graphs)
        pa = (ctypes.c_void_p * len(self._plans))(*[p._h.value for p in self._plans])
        ga = (ctypes.c_void_p * len(self._graphs))(*[g._h.value for g in self._graphs])
        pp = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.npairs = pp.shape[0]
        h = ctypes.c_void_p()
        _check(lib().xm_batch_create(len(self._plans), pa, len(self._graphs), ga, self.npairs,
                                     pp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(h)))
        self._h = h

    def set_tuning(self, window=0, unit=0, warps_per_block=0, blocks_per_sm=0, budget_ms=0, merge_ratio=0):
        t = xm_tuning(window, unit, warps_per_block, blocks_per_sm, budget_ms, merge_ratio)
        _check(lib().xm_batch_set_tuning(self._h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = xm_tuning()
        _check(lib().xm_batch_get_tuning(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in xm_tuning._fields_}

    def run(self, stream=None, graph=False):
        fn = lib().xm_batch_run_graph if graph else lib().xm_batch_run
        _check(fn(self._h, _stream(stream)))

    def counts(self, stream=None):
        out = np.zeros(2 * self.npairs, np.uint64)
        _check(lib().xm_batch_counts(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _stream(stream)))
        lo, hi = out[0::2], out[1::2]
        return [(int(h) << 64) | int(l) for l, h in zip(lo, hi)]

    def set_pair_budget(self, budget_ms: int):
        """Per-pair device-time budget (0: none); see pair_status()."""
        _check(lib().xm_batch_set_pair_budget(self._h, int(budget_ms)))

    def pair_status(self, stream=None):
        """XM_OK or XM_ETIMEOUT per pair, after a run."""
        st = np.zeros(self.npairs, np.int32)
        _check(lib().xm_batch_pair_status(self._h, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          _stream(stream)))
        return st

    def tune(self, candidates, reps=2, stream=None):
        arr = (xm_tuning * len(candidates))(*[xm_tuning(*c) for c in candidates])
        best = xm_tuning()
        ms = ctypes.c_float()
        _check(lib().xm_batch_tune(self._h, arr, len(candidates), reps, ctypes.byref(best), ctypes.byref(ms),
                                   _stream(stream)))
        return {f: getattr(best, f) for f, _ in xm_tuning._fields_}, ms.value

    def free(self):
        if getattr(self, "_h", None):
            lib().xm_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def xm_count_batch(plans, graphs, pairs, stream=None):
    """One-shot batch: exact count of every (plan index, graph index) pair."""
    b = Batch(plans, graphs, pairs)
    try:
        b.run(stream)
        return b.counts(stream)
    finally:
        b.free()


def xm_query_bytes(g: Graph, p: Plan) -> int:
    """Admission estimate (device scratch bytes) of a count query."""
    return int(lib().xm_query_bytes(g._h, p._h))


class Server:
    """Resident graphs + slots; queries are admitted by scratch memory and
    overlap on the GPU (one stream per slot)."""

    def __init__(self, graphs, slots: int = 8, mem_budget_bytes: int = 120 << 30):
        self._graphs = list(graphs)
        ga = (ctypes.c_void_p * len(self._graphs))(*[g._h.value for g in self._graphs])
        h = ctypes.c_void_p()
        _check(lib().xm_server_create(len(self._graphs), ga, slots, mem_budget_bytes, ctypes.byref(h)))
        self._h = h
        self.slots = slots

    def submit(self, plan: Plan, graph_index: int, tag: int) -> bool:
        adm = ctypes.c_int32()
        _check(lib().xm_server_submit(self._h, plan._h, graph_index, tag, ctypes.byref(adm)))
        return bool(adm.value)

    def poll(self, wait: bool = False, max_results: int = 256):
        """[(tag, count or None, status)] of finished queries."""
        tags = (ctypes.c_int64 * max_results)()
        counts = (ctypes.c_uint64 * (2 * max_results))()
        st = (ctypes.c_int32 * max_results)()
        n = ctypes.c_int32()
        _check(lib().xm_server_poll(self._h, 1 if wait else 0, max_results, tags, counts, st, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            c = (counts[2 * i + 1] << 64) | counts[2 * i] if st[i] == XM_OK else None
            out.append((tags[i], c, st[i]))
        return out

    def info(self):
        b, by = ctypes.c_int32(), ctypes.c_uint64()
        _check(lib().xm_server_info(self._h, ctypes.byref(b), ctypes.byref(by)))
        return b.value, by.value

    def free(self):
        if getattr(self, "_h", None):
            lib().xm_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def xm_count_roots(g: Graph, p: Plan, roots, stream=None) -> int:
    """Matches whose start vertex maps to one of `roots` (host int array)."""
    r = np.ascontiguousarray(roots, np.int32)
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().xm_count_roots(g._h, p._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(r),
                                ctypes.byref(lo), ctypes.byref(hi), _stream(stream)))
    return (hi.value << 64) | lo.value


def xm_count_roots_each(g: Graph, p: Plan, roots, stream=None) -> list:
    """Per-start-node counts, in the order of `roots` (host int array)."""
    r = np.ascontiguousarray(roots, np.int32)
    out = np.zeros(2 * max(len(r), 1), np.uint64)
    _check(lib().xm_count_roots_each(g._h, p._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(r),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _stream(stream)))
    return [(int(out[2 * i + 1]) << 64) | int(out[2 * i]) for i in range(len(r))]


def xm_enumerate_roots(g: Graph, p: Plan, roots, out, capacity: int | None = None, stream=None):
    r = np.ascontiguousarray(roots, np.int32)
    cap = out.numel() // p.k if capacity is None else capacity
    total, written = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().xm_enumerate_roots(g._h, p._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(r), _ptr(out),
                                  cap, ctypes.byref(total), ctypes.byref(written), _stream(stream))
    if rc not in (XM_OK, XM_EOVERFLOW):
        _check(rc)
    return total.value, written.value, rc == XM_EOVERFLOW


def xm_count_roots_stats(g: Graph, p: Plan, roots, stream=None):
    r = np.ascontiguousarray(roots, np.int32)
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    st = xm_stats()
    _check(lib().xm_count_roots_stats(g._h, p._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(r),
                                      ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(st), _stream(stream)))
    return (hi.value << 64) | lo.value, {f: getattr(st, f) for f, _ in xm_stats._fields_ if f != "reserved"}


def xm_plan_tune(g: Graph, p: Plan, candidates, reps: int = 2, roots=None, stream=None):
    """Autotune p's launch parameters on graph g (on the counts of a
    start-node list when `roots` is given); returns (best tuning, ms)."""
    arr = (xm_tuning * len(candidates))(*[xm_tuning(*c) for c in candidates])
    best = xm_tuning()
    ms = ctypes.c_float()
    if roots is None:
        _check(lib().xm_plan_tune(g._h, p._h, arr, len(candidates), reps, ctypes.byref(best), ctypes.byref(ms),
                                  _stream(stream)))
    else:
        r = np.ascontiguousarray(roots, np.int32)
        _check(lib().xm_plan_tune_roots(g._h, p._h, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(r), arr,
                                        len(candidates), reps, ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
    return {f: getattr(best, f) for f, _ in xm_tuning._fields_}, ms.value
