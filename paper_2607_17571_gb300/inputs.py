"""Seeded synthetic edge relations (uint32 src/dst pairs).

This module is shared by the oracle tests, the CUDA parity tests and the
benchmark.  It holds no step of the fixpoint method: it only draws graphs.

Every random number comes from one counter-based generator, splitmix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value i of a stream keyed by k is mix(k + (i + 1) * GAMMA).
Being counter-based and written out here in integer arithmetic, it produces
the same graphs on every machine and every numpy version.

Graph families (the shapes of the paper's evaluation workloads, Sec. Evaluation
"Datasets": skewed SNAP graphs, long-fixpoint meshes, family trees):

* ``er_graph``      directed Erdos-Renyi, uniform endpoints, no self-loops,
                    no duplicates, exactly ``n_edges`` distinct edges.
* ``rmat_dag``      R-MAT (a, b, c, d) quadrant recursion, random relabel,
                    only src < dst kept (a DAG), exactly ``n_edges`` edges.
* ``sg_forest``     BFS-grown forest with Poisson(lambda) branching, plus
                    cross edges u -> v between distinct nodes of equal depth.
* ``batch_queries`` the many-small-queries mix: ER graphs with node count
                    log-uniform in [64, 16384] and mean degree U[1.2, 3.0].
* ``serve_request`` the served mix of TC / SG queries of very different sizes,
                    with ``poisson_arrivals`` for an open-loop arrival stream.
* small closed-form families: ``path``, ``cycle``, ``binary_tree``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix_int(x: int) -> int:
    return int(_mix(np.array([x & _MASK64], dtype=np.uint64))[0])


def _tag(name: str) -> int:
    h = 1469598103934665603  # FNV-1a over the tag name
    for ch in name.encode():
        h = ((h ^ ch) * 1099511628211) & _MASK64
    return h


class Stream:
    """A splitmix64 stream keyed by (seed, tag); draws are consumed in order."""

    def __init__(self, seed: int, tag: str):
        self.key = np.uint64(_mix_int((seed * 0x9E3779B97F4A7C15) ^ _tag(tag)))
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _GAMMA)

    def below(self, n: int, bound: int) -> np.ndarray:
        """n integers in [0, bound), bound <= 2**32 (multiply-shift)."""
        hi = self.u64(n) >> np.uint64(32)
        return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.uint64)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class EdgeList:
    src: np.ndarray  # uint32
    dst: np.ndarray  # uint32
    meta: dict

    def __len__(self):
        return int(self.src.shape[0])


def _first_distinct(keys: np.ndarray, count: int):
    """The first ``count`` distinct values of ``keys`` in draw order, or None."""
    uniq, first = np.unique(keys, return_index=True)
    if uniq.shape[0] < count:
        return None
    return keys[np.sort(first)[:count]]


def _split(keys: np.ndarray, meta: dict) -> EdgeList:
    keys = keys.astype(np.uint64)
    return EdgeList((keys >> np.uint64(32)).astype(np.uint32),
                    (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), meta)


def er_graph(n_nodes: int, n_edges: int, seed: int) -> EdgeList:
    """Directed Erdos-Renyi: uniform (src, dst), self-loops and duplicates
    dropped, drawing continues until ``n_edges`` distinct edges exist."""
    if n_edges > n_nodes * (n_nodes - 1):
        raise ValueError("more edges than distinct non-loop pairs")
    s = Stream(seed, "er")
    drawn = np.empty(0, dtype=np.uint64)
    while True:
        m = max(1024, 2 * n_edges)
        a = s.below(m, n_nodes)
        b = s.below(m, n_nodes)
        k = (a << np.uint64(32)) | b
        drawn = np.concatenate([drawn, k[a != b]])
        got = _first_distinct(drawn, n_edges)
        if got is not None:
            return _split(got, dict(family="er", n_nodes=n_nodes, n_edges=n_edges, seed=seed))


def rmat_dag(scale: int, n_edges: int, seed: int, abcd=(0.57, 0.19, 0.19, 0.05)) -> EdgeList:
    """R-MAT quadrant recursion over 2**scale nodes, random node relabel, then
    only edges with src < dst are kept (self-loops and duplicates dropped)
    until ``n_edges`` distinct edges exist."""
    a, b, c, _ = abcd
    n = 1 << scale
    s = Stream(seed, "rmat")
    perm = np.argsort(Stream(seed, "rmat-relabel").u64(n), kind="stable").astype(np.uint64)
    t1, t2, t3 = a, a + b, a + b + c
    drawn = np.empty(0, dtype=np.uint64)
    while True:
        m = max(4096, 3 * n_edges)
        u = s.uniform(m * scale).reshape(m, scale)
        row = ((u >= t2)).astype(np.uint64)                    # quadrants c, d
        col = (((u >= t1) & (u < t2)) | (u >= t3)).astype(np.uint64)  # quadrants b, d
        w = (np.uint64(1) << np.arange(scale - 1, -1, -1, dtype=np.uint64))
        src = perm[(row * w).sum(axis=1, dtype=np.uint64)]
        dst = perm[(col * w).sum(axis=1, dtype=np.uint64)]
        keep = src < dst
        k = (src[keep] << np.uint64(32)) | dst[keep]
        drawn = np.concatenate([drawn, k])
        got = _first_distinct(drawn, n_edges)
        if got is not None:
            return _split(got, dict(family="rmat_dag", scale=scale, n_edges=n_edges, seed=seed,
                                    abcd=list(abcd)))


def rmat_sym(scale: int, n_pairs: int, seed: int, abcd=(0.57, 0.19, 0.19, 0.05)) -> EdgeList:
    """Undirected R-MAT graph as a symmetric edge list: the ``n_pairs``
    distinct pairs u < v of ``rmat_dag`` in both directions (2 * n_pairs
    edges, no self-loops) -- the shape of the undirected graphs triangle
    counting runs on."""
    g = rmat_dag(scale, n_pairs, seed, abcd)
    src = np.concatenate([g.src, g.dst])
    dst = np.concatenate([g.dst, g.src])
    return EdgeList(src, dst, dict(family="rmat_sym", scale=scale, n_pairs=n_pairs, seed=seed,
                                   abcd=list(abcd)))


def rmat_dag16(scale: int, n_edges: int, seed: int, abcd=(0.57, 0.19, 0.19, 0.05)) -> EdgeList:
    """The rmat_dag recipe (quadrant recursion, random relabel, src < dst,
    distinct, exactly ``n_edges``) drawing 16-bit uniforms: one splitmix64
    value decides four levels, so quadrant probabilities have 2^-16
    resolution.  Used for the serving mix, where graphs of up to 10^6 edges
    are drawn on the fly."""
    a, b, c, _ = abcd
    n = 1 << scale
    s = Stream(seed, "rmat16")
    perm = np.argsort(Stream(seed, "rmat16-relabel").u64(n), kind="stable").astype(np.uint64)
    t1, t2, t3 = (int(round(x * 65536)) for x in (a, a + b, a + b + c))
    words = (scale + 3) // 4
    drawn = np.empty(0, dtype=np.uint64)
    while True:
        m = max(4096, 3 * n_edges)
        r = s.u64(m * words).reshape(m, words)
        src = np.zeros(m, dtype=np.int64)
        dst = np.zeros(m, dtype=np.int64)
        for k in range(scale):  # most significant level first
            u = ((r[:, k // 4] >> np.uint64(16 * (k % 4))) & np.uint64(0xFFFF)).astype(np.int64)
            src = (src << 1) | (u >= t2)
            dst = (dst << 1) | (((u >= t1) & (u < t2)) | (u >= t3))
        src = perm[src]
        dst = perm[dst]
        keep = src < dst
        drawn = np.concatenate([drawn, (src[keep] << np.uint64(32)) | dst[keep]])
        got = _first_distinct(drawn, n_edges)
        if got is not None:
            return _split(got, dict(family="rmat_dag16", scale=scale, n_edges=n_edges, seed=seed))


def _poisson_cdf(lam: float, kmax: int = 64):
    p = math.exp(-lam)
    cdf, acc = [], 0.0
    for k in range(kmax):
        acc += p
        cdf.append(acc)
        p *= lam / (k + 1)
    return np.array(cdf)


def sg_forest(n_nodes: int, n_roots: int, lam: float, cross_frac: float, seed: int) -> EdgeList:
    """Forest grown breadth-first from ``n_roots`` roots; node i (in BFS order,
    which is also its id) draws Poisson(lam) children by inversion of its own
    uniform; growth stops at exactly ``n_nodes`` nodes.  Then
    round(cross_frac * tree_edges) distinct cross edges u -> v are added with
    depth(u) == depth(v), u != v.  Edges point parent -> child."""
    s = Stream(seed, "forest")
    cdf = _poisson_cdf(lam)
    depth = np.zeros(n_nodes, dtype=np.int64)
    parents = []
    children = []
    next_id = n_roots
    frontier = np.arange(n_roots, dtype=np.int64)
    d = 0
    while next_id < n_nodes:
        if frontier.shape[0] == 0:
            raise RuntimeError("forest died out before reaching n_nodes")
        u = s.uniform(frontier.shape[0])
        k = np.searchsorted(cdf, u, side="right")
        room = n_nodes - next_id
        csum = np.cumsum(k)
        k = np.minimum(k, np.maximum(0, room - (csum - k)))
        total = int(k.sum())
        par = np.repeat(frontier, k)
        kids = np.arange(next_id, next_id + total, dtype=np.int64)
        parents.append(par)
        children.append(kids)
        depth[kids] = d + 1
        next_id += total
        frontier = kids
        d += 1
    par = np.concatenate(parents) if parents else np.empty(0, np.int64)
    kid = np.concatenate(children) if children else np.empty(0, np.int64)
    n_tree = par.shape[0]
    n_cross = int(round(cross_frac * n_tree))
    # nodes grouped by depth (ids are BFS order, so each level is a contiguous range)
    level_start = np.searchsorted(depth, np.arange(depth.max() + 2), side="left")
    sizes = np.diff(level_start)
    eligible = np.repeat(sizes >= 2, sizes)            # nodes whose level has a partner
    elig_ids = np.nonzero(eligible)[0]
    tree_keys = (par.astype(np.uint64) << np.uint64(32)) | kid.astype(np.uint64)
    cross = np.empty(0, dtype=np.uint64)
    cs = Stream(seed, "forest-cross")
    while cross.shape[0] < n_cross and elig_ids.shape[0] > 0:
        m = max(256, 2 * n_cross)
        uu = elig_ids[cs.below(m, elig_ids.shape[0]).astype(np.int64)]
        lvl = depth[uu]
        lo = level_start[lvl]
        sz = sizes[lvl]
        r = cs.below(m, 2 ** 32).astype(np.int64)
        vv = lo + (r * (sz - 1) >> 32)                   # uniform over the other sz-1 nodes
        vv = vv + (vv >= uu)
        k = (uu.astype(np.uint64) << np.uint64(32)) | vv.astype(np.uint64)
        allk = np.concatenate([cross, k])
        uniq, first = np.unique(allk, return_index=True)
        cross = allk[np.sort(first)][:n_cross]
    keys = np.concatenate([tree_keys, cross])
    return _split(keys, dict(family="sg_forest", n_nodes=n_nodes, n_roots=n_roots, lam=lam,
                             cross_frac=cross_frac, seed=seed, n_tree_edges=int(n_tree),
                             n_cross_edges=int(cross.shape[0]), max_depth=int(depth.max())))


def batch_query_sizes(n_queries: int, seed0: int = 40000, lo: int = 64, hi: int = 16384,
                      deg_lo: float = 1.2, deg_hi: float = 3.0):
    """(n_nodes, n_edges, seed) of each query in the many-small-queries mix:
    n = round(exp(U(ln lo, ln hi))), |E| = round(n * U(deg_lo, deg_hi))."""
    out = []
    for q in range(n_queries):
        s = Stream(seed0 + q, "batch-size")
        u = s.uniform(2)
        n = int(round(math.exp(math.log(lo) + u[0] * (math.log(hi) - math.log(lo)))))
        m = int(round(n * (deg_lo + u[1] * (deg_hi - deg_lo))))
        out.append((n, m, seed0 + q))
    return out


def batch_queries(n_queries: int, seed0: int = 40000, **kw):
    return [er_graph(n, m, s) for (n, m, s) in batch_query_sizes(n_queries, seed0, **kw)]


def serve_request(r: int, seed: int = 5, rmat_edges=(10_000, 1_000_000)):
    """Request r of the served mix: (kind, EdgeList).  TC 75% / SG 25%.  TC
    graphs: 70% ER with the batch mix's sizes, 30% R-MAT DAGs with |E|
    log-uniform in ``rmat_edges`` on 2^ceil(log2(|E|/3)) nodes.  SG graphs:
    the forest recipe (one root per 1,500 nodes, at least 8, Poisson(2) branching, 1%
    equal-depth cross edges) with the batch mix's node counts."""
    st = Stream(seed * 1_000_003 + r, "serve")
    u = st.uniform(4)
    sub = seed * 1_000_003 + r
    n = int(round(math.exp(math.log(64) + u[2] * (math.log(16384) - math.log(64)))))
    if u[0] < 0.25:
        return "sg", sg_forest(max(n, 64), max(8, n // 1500), 2.0, 0.01, sub)
    if u[1] < 0.70:
        return "tc", er_graph(n, int(round(n * (1.2 + u[3] * 1.8))), sub)
    lo, hi = rmat_edges
    m = int(round(math.exp(math.log(lo) + u[3] * (math.log(hi) - math.log(lo)))))
    scale = max(4, math.ceil(math.log2(m / 3)))
    return "tc", rmat_dag16(scale, m, sub)


def poisson_arrivals(n: int, rate: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson stream: exponential gaps."""
    u = Stream(seed, f"arrivals-{rate}").uniform(n)
    return np.cumsum(-np.log1p(-u) / rate)


def path(n: int) -> EdgeList:
    """v0 -> v1 -> ... -> v_{n-1}."""
    i = np.arange(max(n - 1, 0), dtype=np.uint32)
    return EdgeList(i, i + 1, dict(family="path", n=n))


def cycle(n: int) -> EdgeList:
    i = np.arange(n, dtype=np.uint32)
    return EdgeList(i, ((i + 1) % n).astype(np.uint32), dict(family="cycle", n=n))


def binary_tree(depth: int) -> EdgeList:
    """Complete binary tree with levels 0..depth, heap numbering, edges parent -> child."""
    n = (1 << (depth + 1)) - 1
    kid = np.arange(1, n, dtype=np.uint32)
    return EdgeList(((kid - 1) // 2).astype(np.uint32), kid, dict(family="binary_tree", depth=depth))


def random_small(n_nodes: int, n_draws: int, seed: int, allow_loops: bool = True) -> EdgeList:
    """Up to ``n_draws`` uniform edges (duplicates and, optionally, self-loops
    kept in the list; the library treats the input as a set)."""
    s = Stream(seed, "small")
    a = s.below(n_draws, n_nodes).astype(np.uint32)
    b = s.below(n_draws, n_nodes).astype(np.uint32)
    if not allow_loops:
        keep = a != b
        a, b = a[keep], b[keep]
    return EdgeList(a, b, dict(family="random_small", n_nodes=n_nodes, seed=seed))


# The five workloads, by name.  Sizes follow the paper's evaluation scale
# (closures of 10^5..10^8+ tuples, hub degrees in the thousands).
def workload(name: str) -> EdgeList:
    if name == "tc_er_1k":
        return er_graph(1000, 3000, seed=1)
    if name == "tc_rmat17_400k":
        return rmat_dag(17, 400_000, seed=2)
    if name == "sg_forest_60k":
        return sg_forest(60_000, 40, 2.0, 0.01, seed=3)
    if name == "tc_rmat15_100k":  # a smaller skewed case (profiling captures)
        return rmat_dag(15, 100_000, seed=2)
    if name == "tc_rmat19_400k":  # the same recipe on 2^19 nodes: ranks need 17 bits (64-bit keys)
        return rmat_dag(19, 400_000, seed=2)
    if name == "tc_rmat19_150k":  # 64-bit keys at profiling size (76,647 vertices)
        return rmat_dag(19, 150_000, seed=2)
    if name == "tri_rmat16_800k":  # triangle counting: undirected, 800k directed edges
        return rmat_sym(16, 400_000, seed=6)
    raise KeyError(name)
