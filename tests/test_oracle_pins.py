"""Pins of the CPU oracle against facts fixed outside the oracle itself.

* the paper's worked chain example (tests/golden/chain_tc.txt),
* closed forms (path, directed cycle, complete binary tree, forest),
* brute force: BFS shortest walks (TC) and reachability in the pair graph /
  a dense boolean naive fixpoint (SG), exhaustively on every digraph with up
  to 3 nodes (self-loops included) and on random graphs up to 48 nodes.

Each brute-force check also fixes the per-iteration delta sizes: for TC,
Delta^k is exactly the set of pairs at shortest walk length k + 1; for SG,
Delta^k is exactly the set of pairs first reached at breadth-first level k of
the pair graph (equivalently first derived in round k of naive evaluation).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle_sg, oracle_tc, oracle_tc_rows
from paper_2607_17571_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _keys(pairs):
    return np.array(sorted((int(s) << 32) | int(d) for s, d in pairs), dtype=np.uint64)


# --------------------------------------------------------------------------- brute force
def tc_brute(n, edges):
    """Shortest walk length (>= 1) between every ordered pair, by BFS."""
    adj = [[] for _ in range(n)]
    for s, d in set(edges):
        adj[s].append(d)
    dist = {}
    for x in range(n):
        frontier, seen, k = set(adj[x]), set(), 1
        while frontier:
            nxt = set()
            for y in frontier:
                if y in seen:
                    continue
                seen.add(y)
                dist[(x, y)] = k
                nxt.update(adj[y])
            frontier = nxt - seen
            k += 1
    return dist


def check_tc_against_brute(n, edges):
    src = [s for s, _ in edges]
    dst = [d for _, d in edges]
    r = oracle_tc(src, dst)
    dist = tc_brute(n, edges)
    assert r.status == 0
    assert np.array_equal(r.keys, _keys(dist.keys()))
    maxd = max(dist.values(), default=0)
    assert r.iters == max(1, maxd)
    want_log = [sum(1 for v in dist.values() if v == k + 1) for k in range(r.iters + 1)]
    assert r.log.tolist() == want_log
    return r


def sg_pair_graph(n, edges):
    """Pairs reachable in the pair graph: start at (x, y), x != y, children of a
    common p; step (a, b) -> (x, y) along a -> x and b -> y.  Level of first
    reach = iteration of first derivation."""
    ch = [[] for _ in range(n)]
    for s, d in set(edges):
        ch[s].append(d)
    level = {}
    frontier = set()
    for p in range(n):
        for x in ch[p]:
            for y in ch[p]:
                if x != y:
                    frontier.add((x, y))
    k = 0
    while frontier:
        for t in frontier:
            level[t] = k
        nxt = set()
        for a, b in frontier:
            for x in ch[a]:
                for y in ch[b]:
                    if (x, y) not in level:
                        nxt.add((x, y))
        frontier = nxt
        k += 1
    return level


def sg_dense_naive(n, edges):
    """Naive evaluation with boolean matrices: S <- B | A^T S A until stable.
    Returns the list of the per-round new-fact sets."""
    A = np.zeros((n, n), dtype=bool)
    for s, d in edges:
        A[s, d] = True
    Ai = A.astype(np.int64)
    B = (Ai.T @ Ai > 0) & ~np.eye(n, dtype=bool)
    S = B.copy()
    rounds = [B.copy()]
    while True:
        S2 = S | ((Ai.T @ S.astype(np.int64) @ Ai) > 0)
        new = S2 & ~S
        rounds.append(new)
        if not new.any():
            return S, rounds
        S = S2


def check_sg_against_brute(n, edges):
    src = [s for s, _ in edges]
    dst = [d for _, d in edges]
    r = oracle_sg(src, dst)
    level = sg_pair_graph(n, edges)
    assert r.status == 0
    assert np.array_equal(r.keys, _keys(level.keys()))
    maxl = max(level.values(), default=-1)
    assert r.iters == max(1, maxl + 1)
    want_log = [sum(1 for v in level.values() if v == k) for k in range(r.iters + 1)]
    assert r.log.tolist() == want_log
    return r


# --------------------------------------------------------------------------- worked example
def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, *v = line.split()
                out[k] = [int(x) for x in v]
    return out


def test_chain_worked_example():
    g = _read_golden("chain_tc.txt")
    e = g["edges"]
    r = oracle_tc(e[0::2], e[1::2])
    assert r.log.tolist() == g["delta_sizes"]
    assert np.cumsum(r.log).tolist() == g["full_sizes"]
    assert r.iters == g["iterations"][0]
    c = g["closure"]
    assert np.array_equal(r.keys, _keys(zip(c[0::2], c[1::2])))


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 3, 4, 7, 33, 200])
def test_path_closed_form(n):
    g = I.path(n)
    r = oracle_tc(g.src, g.dst)
    assert r.keys.shape[0] == n * (n - 1) // 2
    assert r.iters == n - 1
    assert r.log.tolist() == list(range(n - 1, -1, -1))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 64])
def test_cycle_closed_form(n):
    g = I.cycle(n)
    r = oracle_tc(g.src, g.dst)
    assert r.keys.shape[0] == n * n                       # diagonal included
    assert r.iters == n
    assert r.log.tolist() == [n] * n + [0]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_binary_tree_sg_closed_form(d):
    g = I.binary_tree(d)
    r = oracle_sg(g.src, g.dst)
    assert r.keys.shape[0] == sum((1 << l) * ((1 << l) - 1) for l in range(1, d + 1))
    assert r.iters == d
    # Delta^k: pairs at level l whose lowest common ancestor is k + 1 levels up
    want = [sum((1 << l) * (1 << k) for l in range(k + 1, d + 1)) for k in range(d)] + [0]
    assert r.log.tolist() == want


def test_forest_sg_closed_form():
    g = I.sg_forest(3000, 7, 2.0, 0.0, seed=11)
    r = oracle_sg(g.src, g.dst)
    # no cross edges: pairs of distinct nodes at equal depth in the same tree
    n = int(max(g.src.max(), g.dst.max())) + 1
    parent = np.full(n, -1, dtype=np.int64)
    parent[g.dst] = g.src
    root = np.arange(n)
    depth = np.zeros(n, dtype=np.int64)
    for v in range(n):  # BFS ids: parent id < child id
        if parent[v] >= 0:
            root[v] = root[parent[v]]
            depth[v] = depth[parent[v]] + 1
    _, c = np.unique(root * 4096 + depth, return_counts=True)
    assert r.keys.shape[0] == int((c * (c - 1)).sum())
    assert r.iters == int(depth.max())


# --------------------------------------------------------------------------- exhaustive / random
def test_tc_all_digraphs_up_to_3_nodes():
    for n in (1, 2, 3):
        pairs = [(s, d) for s in range(n) for d in range(n)]
        for mask in range(1 << len(pairs)):
            edges = [p for i, p in enumerate(pairs) if mask >> i & 1]
            check_tc_against_brute(n, edges)


def test_sg_all_digraphs_up_to_3_nodes():
    for n in (1, 2, 3):
        pairs = [(s, d) for s in range(n) for d in range(n)]
        for mask in range(1 << len(pairs)):
            edges = [p for i, p in enumerate(pairs) if mask >> i & 1]
            check_sg_against_brute(n, edges)


@pytest.mark.parametrize("seed", range(12))
def test_tc_random_vs_bfs(seed):
    n = [5, 9, 17, 33, 48][seed % 5]
    g = I.random_small(n, 2 * n + seed, seed)
    check_tc_against_brute(n, list(zip(g.src.tolist(), g.dst.tolist())))


@pytest.mark.parametrize("seed", range(12))
def test_sg_random_vs_pair_graph_and_naive(seed):
    n = [4, 8, 12, 20, 30][seed % 5]
    g = I.random_small(n, n + seed % 7, 100 + seed)
    edges = list(zip(g.src.tolist(), g.dst.tolist()))
    r = check_sg_against_brute(n, edges)
    S, rounds = sg_dense_naive(n, edges)
    assert np.array_equal(r.keys, _keys(zip(*np.nonzero(S))))
    assert r.log.tolist()[: len(rounds)] == [int(x.sum()) for x in rounds][: r.iters + 1]


def test_sg_reconvergent_paths_give_diagonal():
    # p -> u, p -> v, u -> w, v -> w: sg(u,v) from the base rule, then sg(w,w)
    r = oracle_sg([0, 0, 1, 2], [1, 2, 3, 3])
    assert (3 << 32) | 3 in set(r.keys.tolist())
    assert (1 << 32) | 1 not in set(r.keys.tolist())


def test_set_semantics_duplicates_and_self_loops():
    r1 = oracle_tc([5, 5, 5, 7], [7, 7, 5, 9])
    r2 = oracle_tc([5, 5, 7], [7, 5, 9])
    assert np.array_equal(r1.keys, r2.keys) and r1.log.tolist() == r2.log.tolist()
    assert (5 << 32) | 5 in set(r1.keys.tolist())


def test_full_uint32_id_range():
    big = 0xFFFFFFFF
    r = oracle_tc([0, big, 7], [big, 7, 0])
    # a 3-cycle 0 -> big -> 7 -> 0: all 9 pairs
    ids = [0, 7, big]
    assert np.array_equal(r.keys, _keys(itertools.product(ids, ids)))
    assert r.iters == 3


def test_empty_and_no_recursion():
    r = oracle_tc([], [])
    assert r.keys.shape[0] == 0 and r.iters == 1 and r.log.tolist() == [0, 0]
    r = oracle_sg([0], [1])                     # a single child: no sibling pair
    assert r.keys.shape[0] == 0 and r.iters == 1 and r.log.tolist() == [0, 0]


def test_iteration_cap():
    g = I.path(10)
    r = oracle_tc(g.src, g.dst, max_iters=4)
    assert r.status == 1 and r.iters == 4 and r.log.shape[0] == 5


@pytest.mark.parametrize("seed", range(4))
def test_rows_equal_global(seed):
    g = I.er_graph(300, 500 + 40 * seed, seed=seed)
    r = oracle_tc(g.src, g.dst)
    srcs = np.unique(g.src)
    keys, row_len, log_sum, mx = oracle_tc_rows(g.src, g.dst, srcs, n_threads=3)
    assert np.array_equal(keys, r.keys)
    assert mx == r.iters
    assert log_sum[: r.iters + 1].tolist() == r.log.tolist()
    assert int(row_len.sum()) == r.keys.shape[0]
