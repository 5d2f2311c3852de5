"""Triangle counting (Sec. Generalization, "Triangle Counting") through the
C-ABI against the CPU oracle: exact equality of the count.

Covers closed forms (directed 3-cycle, self-loop, undirected triangle,
complete digraphs), random digraphs with duplicates and self-loops, a DAG
(no triangle), the empty relation, hubs (long adjacency lists: deep binary
searches), graphs with many sinks (long runs of empty join slabs), both key
widths, several tiles, and the full-size benchmark graph.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle_triangles
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_17571_gb300 import wg
    c = wg.Context(0)
    yield c
    c.close()


def gpu_count(ctx, src, dst):
    rel = ctx.load(src, dst)
    n = ctx.triangles(rel)
    rel.free()
    return n


def check(ctx, src, dst, threads=1):
    want = oracle_triangles(src, dst, n_threads=threads)
    assert gpu_count(ctx, src, dst) == want
    return want


def test_closed_forms(ctx):
    assert gpu_count(ctx, [0, 1, 2], [1, 2, 0]) == 3
    assert gpu_count(ctx, [5], [5]) == 1
    assert gpu_count(ctx, [0, 1, 2, 1, 2, 0], [1, 2, 0, 0, 1, 2]) == 6
    for n in (3, 9, 40):
        es = list(itertools.permutations(range(n), 2))
        assert gpu_count(ctx, [a for a, _ in es], [b for _, b in es]) == n * (n - 1) * (n - 2)


def test_empty_and_dag(ctx):
    assert gpu_count(ctx, [], []) == 0
    g = I.rmat_dag(12, 20000, 5)
    assert gpu_count(ctx, g.src, g.dst) == 0


@pytest.mark.parametrize("seed", range(5))
def test_random_digraphs(ctx, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 3000))
    m = int(rng.integers(n, 8 * n))
    src, dst = rng.integers(0, n, m), rng.integers(0, n, m)
    src = np.concatenate([src, src[: m // 7]])
    dst = np.concatenate([dst, dst[: m // 7]])
    check(ctx, src, dst)


def test_hub_and_sinks(ctx):
    # a hub joined both ways to 5,000 leaves, a ring over the leaves, and
    # 20,000 edges into sinks: deep probes and long runs of empty slabs
    hub, leaves = 0, np.arange(1, 5001)
    sinks = np.arange(10_000, 30_000)
    src = np.concatenate([np.full(5000, hub), leaves, leaves, np.repeat(leaves[:200], 100)])
    dst = np.concatenate([leaves, np.full(5000, hub), np.roll(leaves, 1), sinks])
    check(ctx, src, dst)


def test_wide_keys(ctx):
    # more than 2^16 distinct vertices: 64-bit packed keys
    rng = np.random.default_rng(7)
    ids = np.unique(rng.integers(0, 1 << 32, 80_000, dtype=np.uint64))[:70_000].astype(np.uint32)
    s, d = rng.integers(0, 70_000, 300_000), rng.integers(0, 70_000, 300_000)
    src = np.concatenate([ids[s], ids[:3], ids[d[:1000]]])
    dst = np.concatenate([ids[d], ids[[1, 2, 0]], ids[s[:1000]]])
    rel = ctx.load(src, dst)
    assert rel.info()["field_bits"] > 16
    n = ctx.triangles(rel)
    rel.free()
    assert n == oracle_triangles(src, dst, n_threads=8)


@pytest.mark.parametrize("scale,pairs", [(10, 3000), (13, 40_000)])
def test_rmat_symmetric(ctx, scale, pairs):
    g = I.rmat_sym(scale, pairs, 11)
    t = check(ctx, g.src, g.dst, threads=8)
    assert t % 6 == 0 and t > 0


def test_benchmark_graph(ctx):
    g = I.workload("tri_rmat16_800k")
    got = gpu_count(ctx, g.src, g.dst)
    assert got % 6 == 0
    assert got == oracle_triangles(g.src, g.dst, n_threads=os.cpu_count() or 8)
