"""Pins of the triangle-counting oracle (Sec. Generalization, "Triangle
Counting": triangle(a,b,c) <- edge(a,b), edge(b,c), edge(c,a)).

The rule's tuples are exactly the closed walks of length 3, so their number
is trace(A^3) of the 0/1 adjacency matrix A of the edge set -- computed here
with an integer matrix product, independent of the oracle's range lookups
and binary searches.  Closed forms fix the special cases: a directed 3-cycle
has 3 tuples (its rotations), a complete digraph on n nodes without loops
n(n-1)(n-2), a self-loop (a,a,a) one, an undirected triangle 6, a DAG none.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle_triangles
from paper_2607_17571_gb300 import inputs as I


def _trace_a3(src, dst, n):
    A = np.zeros((n, n), dtype=np.int64)
    A[np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64)] = 1  # a set: 0/1
    return int(np.trace(A @ A @ A))


def test_every_digraph_on_three_nodes():
    pairs = [(a, b) for a in range(3) for b in range(3)]  # self-loops included
    for mask in range(1 << len(pairs)):
        es = [p for i, p in enumerate(pairs) if mask >> i & 1]
        src = [a for a, _ in es]
        dst = [b for _, b in es]
        assert oracle_triangles(src, dst) == _trace_a3(src, dst, 3), es


@pytest.mark.parametrize("seed", range(6))
def test_random_digraphs_with_duplicates_and_loops(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    m = int(rng.integers(n, 6 * n))
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    src = np.concatenate([src, src[: m // 5]])  # duplicates: a set
    dst = np.concatenate([dst, dst[: m // 5]])
    assert oracle_triangles(src, dst) == _trace_a3(src, dst, n)
    assert oracle_triangles(src, dst, n_threads=4) == oracle_triangles(src, dst)


def test_closed_forms():
    assert oracle_triangles([0, 1, 2], [1, 2, 0]) == 3            # directed 3-cycle
    assert oracle_triangles([0, 1, 2], [2, 0, 1]) == 3
    assert oracle_triangles([7], [7]) == 1                         # (a, a, a)
    assert oracle_triangles([], []) == 0
    und = [(0, 1), (1, 2), (2, 0)]
    src = [a for a, b in und] + [b for a, b in und]
    dst = [b for a, b in und] + [a for a, b in und]
    assert oracle_triangles(src, dst) == 6                         # undirected triangle
    for n in (3, 4, 7, 12):
        es = [(a, b) for a, b in itertools.permutations(range(n), 2)]
        assert oracle_triangles([a for a, _ in es], [b for _, b in es]) == n * (n - 1) * (n - 2)


def test_dag_has_none_and_symmetric_counts_are_multiples_of_six():
    g = I.rmat_dag(8, 600, 3)                                      # src < dst: acyclic
    assert oracle_triangles(g.src, g.dst) == 0
    s = I.rmat_sym(8, 600, 3)
    t = oracle_triangles(s.src, s.dst)
    assert t % 6 == 0 and t > 0
    assert t == _trace_a3(s.src, s.dst, int(max(s.src.max(), s.dst.max())) + 1)


def test_ids_are_labels():
    # relabelling the vertices (full uint32 range) changes nothing
    rng = np.random.default_rng(9)
    src, dst = rng.integers(0, 20, 80), rng.integers(0, 20, 80)
    lab = np.unique(rng.integers(0, 1 << 32, 64, dtype=np.uint64))[:20].astype(np.uint32)
    lab[0], lab[1] = 0, 0xFFFFFFFF  # both ends of the id range
    assert len(np.unique(lab)) == 20
    assert oracle_triangles(lab[src], lab[dst]) == _trace_a3(src, dst, 20)
