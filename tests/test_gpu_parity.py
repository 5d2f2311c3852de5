"""End-to-end parity: the CUDA fixpoint through the C-ABI against the CPU
oracle, bit-exact (result keys, iteration count, per-iteration delta sizes).

Covers the paper's worked example, closed forms, random graphs with
duplicates / self-loops, the full uint32 id range, the empty relation, the
iteration cap, both key widths (32-bit keys when 2 * field bits <= 32,
64-bit otherwise), buffer regrowth, the host-driven loop, and profiling.
"""
import numpy as np
import pytest

from oracle import oracle_sg, oracle_tc
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_17571_gb300 import wg
    c = wg.Context(0)
    yield c
    c.close()


def run(ctx, kind, src, dst, **opts):
    rel = ctx.load(src, dst)
    q = (ctx.tc if kind == "tc" else ctx.sg)(rel, **opts)
    st = q.wait()
    keys, log = q.result(), q.delta_sizes()
    info = rel.info()
    q.free()
    rel.free()
    return keys, st, log, info


def check(ctx, kind, src, dst, **opts):
    want = (oracle_tc if kind == "tc" else oracle_sg)(src, dst)
    keys, st, log, info = run(ctx, kind, src, dst, **opts)
    assert keys.shape == want.keys.shape
    assert np.array_equal(keys, want.keys)
    assert st.iterations == want.iters
    assert log == want.log.tolist()
    assert st.n_tuples == want.keys.shape[0]
    return st, info


def test_chain_worked_example(ctx):
    st, _ = check(ctx, "tc", [0, 1, 2], [1, 2, 3])
    assert st.iterations == 3 and st.n_tuples == 6


@pytest.mark.parametrize("n", [2, 3, 17, 300])
def test_path(ctx, n):
    g = I.path(n)
    check(ctx, "tc", g.src, g.dst)


@pytest.mark.parametrize("n", [1, 2, 5, 100])
def test_cycle(ctx, n):
    g = I.cycle(n)
    check(ctx, "tc", g.src, g.dst)


@pytest.mark.parametrize("d", [1, 2, 3, 8])
def test_binary_tree_sg(ctx, d):
    g = I.binary_tree(d)
    check(ctx, "sg", g.src, g.dst)


@pytest.mark.parametrize("separate", [False, True])
@pytest.mark.parametrize("seed", range(8))
def test_random_small_tc(ctx, seed, separate):
    n = [3, 7, 20, 64, 150, 400, 1000, 2500][seed]
    g = I.random_small(n, int(1.5 * n) + 3, seed)
    check(ctx, "tc", g.src, g.dst, separate_stages=separate)


@pytest.mark.parametrize("separate", [False, True])
@pytest.mark.parametrize("seed", range(8))
def test_random_small_sg(ctx, seed, separate):
    n = [3, 7, 20, 64, 150, 400, 1000, 2500][seed]
    g = I.random_small(n, n + 3, 50 + seed)
    check(ctx, "sg", g.src, g.dst, separate_stages=separate)


@pytest.mark.parametrize("separate", [False, True])
def test_er_1k_workload(ctx, separate):
    g = I.workload("tc_er_1k")
    st, info = check(ctx, "tc", g.src, g.dst, separate_stages=separate)
    assert st.regrows >= 1          # capacities started small: the loop resumed after growing
    assert info["field_bits"] == 10


def test_forest_sg_small(ctx):
    g = I.sg_forest(5000, 6, 2.0, 0.01, seed=21)
    check(ctx, "sg", g.src, g.dst)


@pytest.mark.parametrize("shared", [True, False])
def test_long_runs_of_sink_slabs(ctx, shared):
    """Delta tuples into sinks have empty join slabs.  Here they come in runs
    of 40,000 (longer than the delta tuples of one join-emit tile): one before
    the first candidate, runs between tuples that do produce candidates, and
    one after the last.  The tiles next to a run must emit all their own
    candidates and nothing for the run.  Shared sinks keep 16-bit fields
    (32-bit keys); one sink set per hub needs 18 (64-bit keys)."""
    L = 40_000
    src, dst = [], []
    for h in range(4):
        hub = 10 * h
        src += [hub] * L
        dst += (np.arange(L) + (1 << 20) + (0 if shared else h * L)).tolist()
        if h == 0:
            continue  # sinks only: the leading run
        for j in range(3):
            m = hub + 1 + j  # below the sinks in rank: its slab precedes the hub's run
            src.append(hub)
            dst.append(m)
            for z in range(40):
                t = 1000 + 40 * m + z
                src += [m, t]
                dst += [t, 100000 + t]
    src, dst = np.array(src, np.uint32), np.array(dst, np.uint32)
    st, info = check(ctx, "tc", src, dst)
    assert info["field_bits"] == (16 if shared else 18)
    assert st.iterations == 3


def test_full_id_range(ctx):
    big = 0xFFFFFFFF
    check(ctx, "tc", [0, big, 7, 7], [big, 7, 0, 7])
    check(ctx, "sg", [big, big, 5, 6], [5, 6, 0, big - 1])


def test_duplicates_and_self_loops(ctx):
    check(ctx, "tc", [5, 5, 5, 7, 9, 9], [7, 7, 5, 9, 9, 5])
    check(ctx, "sg", [1, 1, 1, 2, 2], [2, 3, 3, 4, 4])


def test_empty(ctx):
    for kind in ("tc", "sg"):
        keys, st, log, _ = run(ctx, kind, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
        assert keys.shape[0] == 0 and st.iterations == 1 and log == [0, 0]


@pytest.mark.parametrize("separate", [False, True])
def test_wide_keys_u64_path(ctx, separate):
    # > 65536 distinct vertices: 17-bit fields, 64-bit keys
    i = np.arange(40000, dtype=np.uint32)
    src = np.concatenate([2 * i, (2 * i[:500] + 1)])
    dst = np.concatenate([2 * i + 1, 2 * i[1:501]])
    st, info = check(ctx, "tc", src, dst, separate_stages=separate)
    assert info["field_bits"] == 17
    t = I.sg_forest(70000, 20000, 2.0, 0.002, seed=4)
    st, info = check(ctx, "sg", t.src, t.dst, separate_stages=separate)
    assert info["field_bits"] == 17


def test_iteration_cap(ctx):
    from paper_2607_17571_gb300 import wg
    g = I.path(60)
    rel = ctx.load(g.src, g.dst)
    q = ctx.tc(rel, max_iters=10)
    with pytest.raises(wg.WgError) as e:
        q.wait()
    assert e.value.code == wg.WG_E_ITER_CAP
    st = q.poll()
    assert st.state == wg.WG_FAILED and st.iterations == 10
    want = oracle_tc(g.src, g.dst, max_iters=10)
    assert q.delta_sizes() == want.log.tolist()
    q.free()
    rel.free()


def test_host_loop_equals_device_loop(ctx):
    from paper_2607_17571_gb300 import wg
    g = I.er_graph(500, 1200, seed=8)
    a = run(ctx, "tc", g.src, g.dst, loop=wg.WG_LOOP_DEVICE)
    b = run(ctx, "tc", g.src, g.dst, loop=wg.WG_LOOP_HOST)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]


def test_profile_mode(ctx):
    g = I.er_graph(800, 2000, seed=3)
    want = oracle_tc(g.src, g.dst)
    rel = ctx.load(g.src, g.dst)
    q = ctx.tc(rel, profile=True)
    q.wait()
    assert np.array_equal(q.result(), want.keys)
    prof = {p["name"]: p for p in q.profile()}
    assert {"join_count", "join_emit", "sort_pass", "dedup_diff_merge"} <= set(prof)
    assert prof["dedup_diff_merge"]["launches"] == want.iters + 1
    assert all(p["total_ms"] > 0 for p in prof.values())
    q.free()
    rel.free()


def test_repeat_is_deterministic_and_reuses_engine(ctx):
    g = I.er_graph(700, 1600, seed=12)
    rel = ctx.load(g.src, g.dst)
    outs = []
    for _ in range(3):
        q = ctx.tc(rel)
        q.wait()
        outs.append(q.result())
        q.free()
    rel.free()
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_result_into_pinned_buffer(ctx):
    # the reusable page-locked result buffer: same bytes as a fresh array,
    # larger-than-needed buffers return the filled prefix, short ones are refused
    from paper_2607_17571_gb300 import wg
    g = I.er_graph(400, 1200, 21)
    want = oracle_tc(g.src, g.dst)
    src, dst = wg.pinned(len(g.src), np.uint32), wg.pinned(len(g.dst), np.uint32)
    src[:], dst[:] = g.src, g.dst
    rel = ctx.load(src, dst)
    q = ctx.tc(rel)
    q.wait()
    buf = wg.pinned(want.keys.shape[0] + 5)
    got = q.result(out=buf)
    assert got.shape == want.keys.shape and np.array_equal(got, want.keys)
    with pytest.raises(ValueError):
        q.result(out=wg.pinned(want.keys.shape[0] - 1))
    q.free()
    rel.free()


@pytest.mark.parametrize("flags", [dict(loop=1), dict(loop=2),  # WG_LOOP_HOST, WG_LOOP_HOST_STAGED
                                   dict(loop=2, separate_stages=True),
                                   dict(full_width=True), dict(copy_back=True),
                                   dict(full_width=True, copy_back=True),
                                   dict(copy_back=True, separate_stages=True),
                                   dict(hash_join=True), dict(hash_join=True, full_width=True)])
def test_ablation_variants_same_result(ctx, flags):
    # the engineering ablations change the layout or the number of passes,
    # never the result, the iteration count or the per-iteration delta sizes
    for g in (I.er_graph(1000, 3000, 1), I.path(70), I.random_small(300, 900, 5)):
        check(ctx, "tc", g.src, g.dst, **flags)
    f = I.sg_forest(3000, 6, 2.0, 0.01, 8)
    check(ctx, "sg", f.src, f.dst, **flags)
    ids = I.er_graph(400, 1500, 2)
    check(ctx, "tc", ids.src.astype(np.uint64) * 9_999_991 % (1 << 32), ids.dst, **flags)


def test_hash_join_hubs_and_regrowth(ctx):
    # a hub of out-degree 3,000 (one long probe cluster) and tiny initial
    # pools (the pools regrow mid-run; the join must keep using the table)
    hub = np.zeros(3000, dtype=np.uint32)
    leaves = np.arange(1, 3001, dtype=np.uint32)
    g = I.er_graph(3001, 6000, 12)
    src = np.concatenate([hub, g.src])
    dst = np.concatenate([leaves, g.dst])
    check(ctx, "tc", src, dst, hash_join=True, reserve_cand=4096, reserve_full=4096)


@pytest.mark.parametrize("separate", [False, True])
def test_repeated_regrowth_from_tiny_pools(separate):
    # a fresh context: pools start at their minimum and grow several times
    # mid-run; the per-tile arrays (lookback words, splits, mixed-tile lists)
    # must be resized with them -- an SG query whose deltas reach 5e5, then TC
    from paper_2607_17571_gb300 import wg
    with wg.Context(0) as c:
        f = I.sg_forest(2189, 3, 2.0, 0.01, 1020)  # deltas up to 534,518 from 2,208 edges
        st, _ = check(c, "sg", f.src, f.dst, separate_stages=separate,
                      reserve_cand=1, reserve_full=1)
        assert st.regrows >= 2
        for gg in (I.er_graph(900, 2700, 31), I.rmat_dag(11, 6000, 32)):
            check(c, "tc", gg.src, gg.dst, separate_stages=separate, reserve_cand=1,
                  reserve_full=1)


def test_overflow_in_the_first_iteration():
    # SG on a star: the base rule alone makes 1,500 * 1,499 candidates, far
    # over the first pools, so the very first plan kernel stops the run --
    # before any later stage record has been written by a plan kernel -- and
    # the engine grows and starts over (a fresh context: no cached capacities)
    from paper_2607_17571_gb300 import wg
    hub = np.zeros(1500, dtype=np.uint32)
    leaves = np.arange(1, 1501, dtype=np.uint32)
    with wg.Context(0) as c:
        for opts in (dict(), dict(separate_stages=True), dict(side_run="never")):
            st, _ = check(c, "sg", hub, leaves, **opts)
            assert st.n_tuples == 1500 * 1499 and st.regrows >= 1
        st, _ = check(c, "sg", hub, leaves, loop=wg.WG_LOOP_HOST_STAGED)


def test_result_digest_matches_the_oracle(ctx):
    # the device digest of a result equals the digest of the oracle's sorted
    # closure (semi-naive and reachability forms), for both key widths
    from oracle import digest_keys, oracle_tc_reach
    for g in (I.er_graph(500, 1500, 21), I.rmat_dag(11, 5000, 22), I.cycle(40)):
        rel = ctx.load(g.src, g.dst)
        q = ctx.tc(rel)
        q.wait()
        want = oracle_tc(g.src, g.dst)
        n, iters, log, dg = oracle_tc_reach(g.src, g.dst, n_threads=2)
        assert q.digest() == digest_keys(want.keys) == dg
        assert q.digest() == digest_keys(q.result())
        q.free()
        rel.free()
    wide = I.er_graph(100_000, 90_000, 23)  # > 2^16 vertices: 17-bit ranks, 64-bit keys
    rel = ctx.load(wide.src, wide.dst)
    assert rel.info()["field_bits"] > 16
    q = ctx.tc(rel)
    q.wait()
    assert q.digest() == digest_keys(oracle_tc(wide.src, wide.dst).keys)
    q.free()
    rel.free()
    f = I.sg_forest(2500, 5, 2.0, 0.01, 24)
    rel = ctx.load(f.src, f.dst)
    q = ctx.sg(rel)
    q.wait()
    assert q.digest() == digest_keys(oracle_sg(f.src, f.dst).keys)
    q.free()
    rel.free()
