"""CPU oracle for directed subgraph matching -- test infrastructure only.

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package. The GPU library never does, and the two
share no code: the oracle is a plain single-threaded backtracking matcher
over the original (unreduced) pattern, written from the definitions of the
XMiner paper (Sec. 2: Defs. 2.1-2.2 and the vertex/edge constraints), in C
(``xm_oracle.c``), compiled with gcc on first use.

What it computes (see the C file header for the full statement):
  * embeddings: injective maps m with (m(u), m(v)) an arc for every pattern
    arc (u, v) -- non-induced matching;
  * matches: embeddings modulo Aut(P), represented by the orbit-smallest
    tuple; #matches = #embeddings / |Aut(P)|;
  * with induced=True, non-arcs of the pattern must be non-arcs among the
    matched nodes (induced subgraph isomorphism).

Parity pins for every function here live in ``tests/test_oracle.py``
(brute force over all node tuples, closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2, no OpenMP: the oracle is single-threaded)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        u64ref = ctypes.POINTER(ctypes.c_uint64)
        lib.og_build.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p]
        lib.og_build.restype = ctypes.c_void_p
        lib.og_free.argtypes = [ctypes.c_void_p]
        lib.og_free.restype = None
        lib.og_num_arcs.argtypes = [ctypes.c_void_p]
        lib.og_num_arcs.restype = ctypes.c_int64
        lib.og_out_csr.argtypes = [ctypes.c_void_p, i64p, i32p]
        lib.og_out_csr.restype = None
        lib.og_has_arc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        lib.og_has_arc.restype = ctypes.c_int
        lib.og_aut.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_void_p]
        lib.og_aut.restype = ctypes.c_int
        lib.og_count_embeddings.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i32p, i32p,
                                            ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, u64ref, u64ref]
        lib.og_count_embeddings.restype = ctypes.c_int
        lib.og_count_embeddings_capped.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i32p, i32p,
                                                   ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                                   ctypes.c_uint64, u64ref, u64ref]
        lib.og_count_embeddings_capped.restype = ctypes.c_int
        lib.og_count_matches.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int,
                                         u64ref, u64ref]
        lib.og_count_matches.restype = ctypes.c_int
        lib.og_enumerate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int64]
        lib.og_enumerate.restype = ctypes.c_int64
        lib.og_canonicalize.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int64, i32p, i32p]
        lib.og_canonicalize.restype = None
        lib.og_enumerate_embeddings.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_int64]
        lib.og_enumerate_embeddings.restype = ctypes.c_int64
        lib.og_triangle_sums.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, u64ref, u64ref]
        lib.og_triangle_sums.restype = None
        _lib = lib
    return _lib


def _pattern_arrays(pattern):
    k, arcs = pattern
    ps = np.array([a for a, _ in arcs], np.int32)
    pd = np.array([b for _, b in arcs], np.int32)
    return k, len(arcs), ps, pd


def automorphisms(pattern) -> np.ndarray:
    """All automorphisms of the pattern as rows s with s[v] = image of v."""
    k, e, ps, pd = _pattern_arrays(pattern)
    buf = np.empty(40320 * k, np.int32)
    cnt = _L().og_aut(k, e, ps, pd, buf.ctypes.data)
    if cnt < 0:
        raise ValueError("pattern too large for the oracle (k <= 8)")
    return buf[: cnt * k].reshape(cnt, k).copy()


class OracleGraph:
    """Deduplicated digraph (self-loops dropped) with sorted out- and in-lists."""

    def __init__(self, n: int, src: np.ndarray, dst: np.ndarray):
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        self.n = int(n)
        self._h = _L().og_build(self.n, len(src), src, dst)
        if not self._h:
            raise ValueError("og_build failed (bad node id or out of memory)")
        self.m = int(_L().og_num_arcs(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.og_free(h)
            self._h = None

    def out_csr(self):
        off = np.empty(self.n + 1, np.int64)
        adj = np.empty(max(self.m, 1), np.int32)
        _L().og_out_csr(self._h, off, adj)
        return off, adj[: self.m]

    def has_arc(self, u: int, v: int) -> bool:
        return bool(_L().og_has_arc(self._h, u, v))

    def count_embeddings(self, pattern, root: int = 0, r_lo: int = 0, r_hi: int | None = None,
                         induced: bool = False) -> int:
        """Embeddings m with m(root) in [r_lo, r_hi) (induced: non-arcs too)."""
        k, e, ps, pd = _pattern_arrays(pattern)
        lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
        r_hi = self.n if r_hi is None else r_hi
        if _L().og_count_embeddings(self._h, k, e, ps, pd, root, r_lo, r_hi, int(induced), ctypes.byref(lo),
                                    ctypes.byref(hi)):
            raise ValueError("bad pattern")
        return (hi.value << 64) | lo.value

    def count_embeddings_capped(self, pattern, root: int, r_lo: int, r_hi: int, max_steps: int,
                                induced: bool = False):
        """count_embeddings, or None when the walk would examine more than
        max_steps candidates."""
        k, e, ps, pd = _pattern_arrays(pattern)
        lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
        rc = _L().og_count_embeddings_capped(self._h, k, e, ps, pd, root, r_lo, r_hi, int(induced), max_steps,
                                             ctypes.byref(lo), ctypes.byref(hi))
        if rc < 0:
            raise ValueError("bad pattern")
        return None if rc == 1 else (hi.value << 64) | lo.value

    def count_matches(self, pattern, induced: bool = False) -> int:
        """Distinct matched subgraphs (orbit-smallest embeddings)."""
        k, e, ps, pd = _pattern_arrays(pattern)
        lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
        if _L().og_count_matches(self._h, k, e, ps, pd, int(induced), ctypes.byref(lo), ctypes.byref(hi)):
            raise ValueError("bad pattern")
        return (hi.value << 64) | lo.value

    def enumerate(self, pattern, capacity: int | None = None, induced: bool = False) -> np.ndarray:
        """All matches as an (N, k) int32 array, each row the orbit-smallest
        embedding in pattern-vertex order, rows sorted lexicographically."""
        k, e, ps, pd = _pattern_arrays(pattern)
        if capacity is None:
            capacity = int(_L().og_enumerate(self._h, k, e, ps, pd, int(induced), None, 0))
        buf = np.empty(max(capacity, 1) * k, np.int32)
        total = int(_L().og_enumerate(self._h, k, e, ps, pd, int(induced), buf.ctypes.data, capacity))
        rows = buf[: min(total, capacity) * k].reshape(-1, k)
        return sort_rows(rows)


    def enumerate_embeddings(self, pattern, root: int = 0, r_lo: int = 0, r_hi: int | None = None,
                             induced: bool = False) -> np.ndarray:
        """Every embedding m with m(root) in [r_lo, r_hi), as an (N, k) int32
        array in pattern-vertex order, rows sorted lexicographically."""
        k, e, ps, pd = _pattern_arrays(pattern)
        r_hi = self.n if r_hi is None else r_hi
        total = int(_L().og_enumerate_embeddings(self._h, k, e, ps, pd, root, r_lo, r_hi, int(induced), None, 0))
        if total < 0:
            raise ValueError("bad pattern")
        buf = np.empty(max(total, 1) * k, np.int32)
        _L().og_enumerate_embeddings(self._h, k, e, ps, pd, root, r_lo, r_hi, int(induced), buf.ctypes.data, total)
        return sort_rows(buf[: total * k].reshape(-1, k))

    def triangle_sums(self, u_lo: int = 0, u_hi: int | None = None):
        """(feed-forward triangles, closed 3-walks) over the arcs whose source
        is in [u_lo, u_hi): over all nodes sum(A o A^2) and tr(A^3)."""
        f, c = ctypes.c_uint64(), ctypes.c_uint64()
        _L().og_triangle_sums(self._h, u_lo, self.n if u_hi is None else u_hi, ctypes.byref(f), ctypes.byref(c))
        return f.value, c.value


def canonicalize(pattern, tuples: np.ndarray) -> np.ndarray:
    """Map each embedding (row, pattern-vertex order) to the smallest tuple of
    its Aut-orbit, then sort the rows."""
    k = pattern[0]
    aut = np.ascontiguousarray(automorphisms(pattern), np.int32)
    t = np.ascontiguousarray(tuples, np.int32).reshape(-1, k)
    out = np.empty_like(t)
    _L().og_canonicalize(k, aut.shape[0], aut.reshape(-1), t.shape[0], t.reshape(-1), out.reshape(-1))
    return sort_rows(out)


def sort_rows(rows: np.ndarray) -> np.ndarray:
    if rows.size == 0:
        return rows.reshape(0, rows.shape[1] if rows.ndim == 2 else 0)
    order = np.lexsort(rows.T[::-1])
    return rows[order]
