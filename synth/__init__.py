"""Seeded synthetic inputs shared by the oracle and the GPU path.

Nothing here matches patterns: it draws data digraphs (directed
Erdos-Renyi, R-MAT) and pattern digraphs, and names the fixed patterns the
workloads use. The C generators live in ``gen.c`` (splitmix64 seeding,
xoshiro256** streams) and are compiled on first use into ``libsynth.so``
next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-march=x86-64-v2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.synth_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
        lib.synth_er.restype = ctypes.c_int
        lib.synth_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.synth_rmat.restype = ctypes.c_int
        lib.synth_trim.argtypes = [ctypes.c_int64, ctypes.c_int32, i32p, i32p]
        lib.synth_trim.restype = ctypes.c_int64
        lib.synth_pattern.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                      i32p, i32p]
        lib.synth_pattern.restype = ctypes.c_int
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, f64p]
        lib.synth_uniform.restype = None
        _lib = lib
    return _lib


# ----------------------------------------------------------------- graphs --

def er_graph(n: int, m: int, seed: int):
    """Directed G(n, m): exactly m distinct arcs u->v, u != v, uniform over
    the n(n-1) ordered pairs. Returns (n, src, dst) as int32 arrays."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _L().synth_er(n, m, seed, src, dst) != 0:
        raise ValueError(f"synth_er failed for n={n} m={m}")
    return n, src, dst


RMAT_ABC = (0.57, 0.19, 0.19)   # d = 0.05


def rmat_graph(scale: int, edge_factor: int, seed: int, a=RMAT_ABC[0], b=RMAT_ABC[1], c=RMAT_ABC[2],
               n_keep: int | None = None):
    """R-MAT digraph with 2^scale nodes and edge_factor * 2^scale drawn arcs
    (repeats and self-loops still present; graph loaders drop them).
    With n_keep, node ids >= n_keep are trimmed away. Returns (n, src, dst)."""
    n_arcs = edge_factor << scale
    src = np.empty(n_arcs, np.int32)
    dst = np.empty(n_arcs, np.int32)
    if _L().synth_rmat(scale, n_arcs, a, b, c, seed, src, dst) != 0:
        raise ValueError("synth_rmat failed")
    n = 1 << scale
    if n_keep is not None and n_keep < n:
        kept = _L().synth_trim(n_arcs, n_keep, src, dst)
        src, dst, n = src[:kept].copy(), dst[:kept].copy(), n_keep
    return n, src, dst


def uniforms(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    _L().synth_uniform(seed, stream, count, out)
    return out


def random_pattern(k: int, rho: float, seed: int, stream: int):
    """Weakly connected random pattern: each ordered pair an arc w.p. rho."""
    ps = np.empty(k * k, np.int32)
    pd = np.empty(k * k, np.int32)
    e = _L().synth_pattern(k, rho, seed, stream, ps, pd)
    if e < 0:
        raise ValueError("synth_pattern failed")
    return k, [(int(ps[i]), int(pd[i])) for i in range(e)]


# --------------------------------------------------------------- patterns --
# Pattern vertices are 0..k-1 as written; arcs are (source, destination).

CYCLE3 = (3, [(0, 1), (1, 2), (2, 0)])                      # directed 3-cycle (3_p)
FFL = (3, [(0, 1), (0, 2), (1, 2)])                         # feed-forward triangle a->b, a->c, b->c
BIFAN = (4, [(0, 2), (1, 2), (0, 3), (1, 3)])               # "rectangle" / bi-fan a->c, b->c, a->d, b->d
CYCLE4 = (4, [(0, 1), (1, 2), (2, 3), (3, 0)])              # directed 4-cycle (4_p)
BIPARALLEL = (4, [(0, 1), (0, 2), (1, 3), (2, 3)])          # a->b, a->c, b->d, c->d
# two feed-forward triangles sharing c (a->b, b->c, a->c; c->d, d->e, c->e) plus the reciprocal b->a
FFCHAIN5 = (5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4), (1, 0)])

# The 13 weakly connected 3-node digraphs up to isomorphism, named by the
# triad census (MAN codes).
MOTIFS3 = {
    "021D": (3, [(1, 0), (1, 2)]),
    "021U": (3, [(0, 1), (2, 1)]),
    "021C": (3, [(0, 1), (1, 2)]),
    "111D": (3, [(0, 1), (1, 0), (2, 1)]),
    "111U": (3, [(0, 1), (1, 0), (1, 2)]),
    "030T": (3, [(0, 1), (2, 1), (0, 2)]),
    "030C": (3, [(0, 1), (1, 2), (2, 0)]),
    "201": (3, [(0, 1), (1, 0), (1, 2), (2, 1)]),
    "120D": (3, [(1, 0), (1, 2), (0, 2), (2, 0)]),
    "120U": (3, [(0, 1), (2, 1), (0, 2), (2, 0)]),
    "120C": (3, [(0, 1), (1, 2), (0, 2), (2, 0)]),
    "210": (3, [(0, 1), (1, 2), (2, 1), (0, 2), (2, 0)]),
    "300": (3, [(0, 1), (1, 0), (1, 2), (2, 1), (0, 2), (2, 0)]),
}

# ------------------------------------------------------ workload recipes --
# Seeds follow the workload table: tiny ER seed 1, R-MAT s20 seed 2,
# R-MAT s24 seed 3.

def tiny_er():
    """Directed ER graph: 2,000 nodes, exactly 20,000 distinct arcs, seed 1."""
    return er_graph(2000, 20000, seed=1)


def rmat20():
    """R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19 d=.05, seed 2."""
    return rmat_graph(20, 16, seed=2)


def rmat24():
    """R-MAT scale 24, edge factor 16, a=.57 b=.19 c=.19 d=.05, seed 3."""
    return rmat_graph(24, 16, seed=3)


TINY_PATTERNS = {"cycle3": CYCLE3, "ffl": FFL, "bifan": BIFAN}
S24_PATTERNS = {"cycle4": CYCLE4, "bifan": BIFAN, "biparallel": BIPARALLEL, "ffchain5": FFCHAIN5}

# patterns whose counts stop early: leaf products (arc-free trailing
# vertices) and cut-vertex splits
LEAF_PRODUCT_PATTERNS = {
    "out_star4": (4, [(0, 1), (0, 2), (0, 3)]),
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "mixed_star4": (4, [(0, 1), (2, 0), (0, 3)]),
    "out_star5": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
}
# denser 5-7-vertex patterns with many inclusion relations (the paper's
# 5-7-vertex patterns are not available): transitive tournaments (every
# arc i -> j for i < j) and complete bipartite fans (every arc u -> v from
# the first group to the second)
def transitive_tournament(k: int):
    return k, [(i, j) for i in range(k) for j in range(i + 1, k)]


def bipartite_fan(a: int, b: int):
    return a + b, [(i, a + j) for i in range(a) for j in range(b)]


DENSE_PATTERNS = {
    "tt5": transitive_tournament(5),
    "tt6": transitive_tournament(6),
    "tt7": transitive_tournament(7),
    "fan24": bipartite_fan(2, 4),
    "fan33": bipartite_fan(3, 3),
}

SPLIT_PATTERNS = {
    "ffchain5": FFCHAIN5,
    "tri_tail": (5, [(0, 1), (1, 2), (0, 2), (2, 3), (2, 4)]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
}


# ------------------------------------------------------ batch / serve recipes

def rmat_graph_arcs(scale: int, n_arcs: int, seed: int, n_keep: int | None = None):
    """R-MAT with an explicit number of drawn arcs (default a, b, c)."""
    src = np.empty(n_arcs, np.int32)
    dst = np.empty(n_arcs, np.int32)
    if _L().synth_rmat(scale, n_arcs, RMAT_ABC[0], RMAT_ABC[1], RMAT_ABC[2], seed, src, dst) != 0:
        raise ValueError("synth_rmat failed")
    n = 1 << scale
    if n_keep is not None and n_keep < n:
        kept = _L().synth_trim(n_arcs, n_keep, src, dst)
        src, dst, n = src[:kept].copy(), dst[:kept].copy(), n_keep
    return n, src, dst


def small_graph(i: int, seed: int, n_lo: int = 50, n_hi: int = 5000):
    """Graph i of a batch: n log-uniform in [n_lo, n_hi], mean out-degree
    uniform in [4, 12], even i: directed ER, odd i: R-MAT on 2^ceil(log2 n)
    nodes trimmed to n (about n * degree arcs kept)."""
    u = uniforms(seed, 10_000_000 + i, 2)
    n = int(round(np.exp(np.log(n_lo) + u[0] * (np.log(n_hi) - np.log(n_lo)))))
    deg = 4.0 + 8.0 * u[1]
    m = min(int(round(n * deg)), n * (n - 1))
    if i % 2 == 0:
        return er_graph(n, m, seed=seed * 1_000_003 + i)
    scale = max(1, int(np.ceil(np.log2(n))))
    # arcs landing inside [0, n)^2 are about a fraction (n / 2^scale)^2 of all (lower for skewed R-MAT);
    # draw enough that about m survive the trim
    frac = (n / float(1 << scale)) ** 2
    return rmat_graph_arcs(scale, int(m / max(frac, 0.05)), seed * 1_000_003 + i, n_keep=n)


def batch_pattern(i: int, seed: int, k_lo: int = 3, k_hi: int = 6):
    """Pattern i of a batch: k uniform in [k_lo, k_hi], arc density rho
    uniform in [0.3, 0.7], redrawn until weakly connected."""
    u = uniforms(seed, 20_000_000 + i, 2)
    k = k_lo + int(u[0] * (k_hi - k_lo + 1))
    return random_pattern(min(k, k_hi), 0.3 + 0.4 * u[1], seed, 30_000_000 + i)
