"""The seeded generators: determinism, exact sizes and the structure each
workload promises (no self-loops/duplicates, DAG orientation, equal-depth
cross edges, log-uniform batch sizes)."""
import hashlib

import numpy as np

from paper_2607_17571_gb300 import inputs as I


def _digest(g):
    return hashlib.sha256(g.src.astype("<u4").tobytes() + g.dst.astype("<u4").tobytes()).hexdigest()


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published generator
    s = I.Stream.__new__(I.Stream)
    s.key = np.uint64(0)
    s.pos = 0
    assert s.u64(3).tolist() == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_determinism():
    assert _digest(I.er_graph(1000, 3000, 1)) == _digest(I.er_graph(1000, 3000, 1))
    assert _digest(I.er_graph(1000, 3000, 1)) != _digest(I.er_graph(1000, 3000, 2))
    assert _digest(I.sg_forest(5000, 4, 2.0, 0.01, 3)) == _digest(I.sg_forest(5000, 4, 2.0, 0.01, 3))


def _check_set(g):
    k = (g.src.astype(np.uint64) << np.uint64(32)) | g.dst
    assert np.unique(k).shape[0] == k.shape[0]
    assert not np.any(g.src == g.dst)


def test_er_exact_size():
    g = I.er_graph(1000, 3000, seed=1)
    assert len(g) == 3000 and g.src.max() < 1000 and g.dst.max() < 1000
    _check_set(g)


def test_rmat_dag_small():
    g = I.rmat_dag(12, 8000, seed=5)
    assert len(g) == 8000
    _check_set(g)
    assert np.all(g.src < g.dst)
    deg = np.bincount(g.src)
    assert deg.max() > 20 * deg[deg > 0].mean() / 4  # skewed: hubs well above the mean


def test_forest_structure():
    g = I.sg_forest(6000, 5, 2.0, 0.01, seed=7)
    m = g.meta
    assert m["n_tree_edges"] == 6000 - 5
    assert m["n_cross_edges"] == round(0.01 * (6000 - 5))
    _check_set(g)
    tree_src, tree_dst = g.src[: m["n_tree_edges"]], g.dst[: m["n_tree_edges"]]
    depth = np.zeros(6000, dtype=np.int64)
    for s, d in zip(tree_src.tolist(), tree_dst.tolist()):
        depth[d] = depth[s] + 1
    # every non-root has exactly one tree parent; cross edges join equal depths
    assert np.bincount(tree_dst, minlength=6000)[5:].tolist() == [1] * (6000 - 5)
    cs, cd = g.src[m["n_tree_edges"]:], g.dst[m["n_tree_edges"]:]
    assert np.all(depth[cs] == depth[cd]) and np.all(cs != cd)


def test_batch_sizes():
    qs = I.batch_query_sizes(4096)
    n = np.array([q[0] for q in qs])
    m = np.array([q[1] for q in qs])
    assert n.min() >= 64 and n.max() <= 16384
    assert np.all(m >= np.round(1.2 * n) - 1) and np.all(m <= np.round(3.0 * n) + 1)
    # log-uniform: the median sits near sqrt(64 * 16384) = 1024
    assert 700 < np.median(n) < 1500


def test_rmat_sym_is_symmetric_loop_free_and_distinct():
    g = I.rmat_sym(10, 2000, 4)
    assert len(g) == 4000
    k = (g.src.astype(np.uint64) << np.uint64(32)) | g.dst
    assert len(np.unique(k)) == 4000 and not np.any(g.src == g.dst)
    rev = (g.dst.astype(np.uint64) << np.uint64(32)) | g.src
    assert np.array_equal(np.sort(k), np.sort(rev))
