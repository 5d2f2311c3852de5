"""Pins of oracle_tc_reach (TC by reachability, with a digest of the sorted
closure) and of the digest itself, on the CPU.

* digest_keys: the digest is a sum of SplitMix64 outputs (Steele, Lea, Flood
  2014); on an all-zero key array its terms are exactly the published
  outputs of SplitMix64 seeded with 0 (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
  0x06C45D188009454F).
* oracle_tc_reach against the brute-force shortest walks of every digraph on
  at most 3 nodes (all self-loop patterns included), against the semi-naive
  oracle_tc on random graphs with duplicates, self-loops and cycles, and
  against the closed forms of a path and a cycle.
"""
import itertools

import numpy as np
import pytest

from oracle import digest_keys, oracle_tc, oracle_tc_reach
from paper_2607_17571_gb300 import inputs as I

SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
M = (1 << 64) - 1


def test_digest_terms_are_the_published_splitmix64_outputs():
    # term i of a zero array is mix64(i * phi): mix64(0) = 0, then the
    # generator's outputs for seed 0 in order
    assert digest_keys(np.zeros(1, dtype=np.uint64)) == 0
    acc = 0
    for k, out in enumerate(SPLITMIX64_SEED0, start=2):
        acc = (acc + out) & M
        assert digest_keys(np.zeros(k, dtype=np.uint64)) == acc


def test_digest_depends_on_order_and_values():
    a = np.array([1, 2, 3], dtype=np.uint64)
    assert digest_keys(a) != digest_keys(a[::-1].copy())
    assert digest_keys(a) != digest_keys(np.array([1, 2, 4], dtype=np.uint64))


def _brute(n, edges):
    adj = [[] for _ in range(n)]
    for s, d in set(edges):
        adj[s].append(d)
    dist = {}
    for x in range(n):
        frontier, seen, k = set(adj[x]), set(), 1
        while frontier:
            nxt = set()
            for y in frontier:
                if y not in seen:
                    seen.add(y)
                    dist[(x, y)] = k
                    nxt.update(adj[y])
            frontier = nxt - seen
            k += 1
    return dist


def _keys(pairs):
    return np.array(sorted((int(s) << 32) | int(d) for s, d in pairs), dtype=np.uint64)


def test_reach_all_digraphs_up_to_3_nodes():
    for n in (1, 2, 3):
        pairs = [(s, d) for s in range(n) for d in range(n)]
        for mask in range(1 << len(pairs)):
            edges = [p for i, p in enumerate(pairs) if mask >> i & 1]
            dist = _brute(n, edges)
            cnt, iters, log, dg = oracle_tc_reach([s for s, _ in edges], [d for _, d in edges])
            assert cnt == len(dist)
            maxd = max(dist.values(), default=0)
            assert iters == max(1, maxd)
            assert log.tolist() == [sum(1 for v in dist.values() if v == k + 1)
                                    for k in range(iters + 1)]
            assert dg == digest_keys(_keys(dist.keys()))


@pytest.mark.parametrize("seed", range(10))
def test_reach_equals_semi_naive(seed):
    n = [6, 20, 60, 200, 700][seed % 5]
    g = I.random_small(n, 3 * n + seed, 500 + seed)  # duplicates and self-loops
    r = oracle_tc(g.src, g.dst)
    for threads in (1, 3):
        cnt, iters, log, dg = oracle_tc_reach(g.src, g.dst, n_threads=threads)
        assert cnt == r.keys.shape[0] and iters == r.iters
        assert log.tolist() == r.log.tolist()
        assert dg == digest_keys(r.keys)


def test_reach_sparse_ids_and_er():
    g = I.er_graph(400, 1200, 3)
    src = g.src.astype(np.uint64) * 10_000_019 % (1 << 32)  # ids over the uint32 range
    r = oracle_tc(src, g.dst)
    cnt, iters, log, dg = oracle_tc_reach(src, g.dst, n_threads=2)
    assert (cnt, iters, log.tolist(), dg) == (r.keys.shape[0], r.iters, r.log.tolist(),
                                             digest_keys(r.keys))


@pytest.mark.parametrize("n", [1, 2, 9, 64])
def test_reach_path_and_cycle_closed_forms(n):
    p = I.path(n)
    cnt, iters, log, _ = oracle_tc_reach(p.src, p.dst)
    assert cnt == n * (n - 1) // 2 and iters == max(1, n - 1)
    c = I.cycle(n)
    cnt, iters, _, dg = oracle_tc_reach(c.src, c.dst)
    assert cnt == n * n and iters == n
    assert dg == digest_keys(_keys(itertools.product(range(n), range(n))))


def test_reach_empty():
    cnt, iters, log, dg = oracle_tc_reach([], [])
    assert (cnt, iters, log.tolist(), dg) == (0, 1, [0, 0], 0)
