"""The library's host CSR build (dual sorted CSR, repeats and self-loops
dropped; the untimed graph preparation) against the oracle's own adjacency,
on the CPU: a small driver compiled with g++ from the library's source runs
several builds in a row (large, tiny, empty, large again) so that staging
buffers reused between builds are covered too."""
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2404_11105_b300", "csrc")


def _cuda_include():
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("cuda_runtime.h not found")
    exe = str(tmp_path_factory.mktemp("csr") / "host_csr")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                           f"-I{inc}", "-o", exe, os.path.join(HERE, "host_csr_main.cpp"),
                           os.path.join(CSRC, "xm_graph_host.cpp")])
    return exe


def _cases():
    rng = np.random.default_rng(11)
    cases = [synth.rmat_graph(14, 8, seed=3)]
    n = 7
    src = rng.integers(0, n, 60).astype(np.int32)
    dst = rng.integers(0, n, 60).astype(np.int32)
    cases.append((n, src, dst))                                       # dense, repeats, loops
    cases.append((1, np.zeros(0, np.int32), np.zeros(0, np.int32)))   # one node, no arcs
    cases.append((3, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32)))  # only loops
    cases.append(synth.er_graph(5000, 60000, seed=4))
    cases.append(synth.rmat_graph(12, 16, seed=5))
    return cases


def test_host_csr_matches_oracle(driver, tmp_path):
    cases = _cases()
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        for n, src, dst in cases:
            f.write(np.array([n, len(src)], np.int64).tobytes())
            f.write(np.ascontiguousarray(src, np.int32).tobytes())
            f.write(np.ascontiguousarray(dst, np.int32).tobytes())
    subprocess.check_call([driver, str(fin), str(fout)])
    buf = open(fout, "rb").read()
    pos = 0

    def take(dtype, count):
        nonlocal pos
        a = np.frombuffer(buf, dtype, count, pos)
        pos += a.nbytes
        return a

    for n, src, dst in cases:
        rc, arcs = take(np.int64, 2)
        assert rc == 0
        out_off, out_adj = take(np.int32, n + 1), take(np.int32, arcs)
        in_off, in_adj = take(np.int32, n + 1), take(np.int32, arcs)
        og = oracle.OracleGraph(n, src, dst)
        ref_off, ref_adj = og.out_csr()
        assert arcs == og.m
        assert np.array_equal(out_off, ref_off) and np.array_equal(out_adj, ref_adj)
        # in-lists: the transpose of the oracle's out-lists, rows ascending
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(ref_off))
        order = np.lexsort((rows, ref_adj))
        want_adj = rows[order].astype(np.int32)
        want_off = np.concatenate([[0], np.cumsum(np.bincount(ref_adj, minlength=n))]).astype(np.int32)
        assert np.array_equal(in_off, want_off) and np.array_equal(in_adj, want_adj)
    assert pos == len(buf)
