"""The full relation as a main run plus a side run of the newest tuples
(single queries, fused stages).

An iteration with few candidates finds its new tuples against both runs and
merges them into the side run only; the side run is folded back into the main
run when it outgrows its pool or the candidates grow again, and the final
relation is the two runs merged.  None of this may change the result, the
iteration count or the per-iteration delta sizes: each case is checked against
the oracle, bit for bit, with the side run off ("never": the disjoint merge
every iteration), in its default policy ("auto") and forced into every
iteration it fits ("always") -- which also makes the side run outgrow its pool
and be folded back several times (the pool holds an eighth of the Full
pool's keys).
"""
import numpy as np
import pytest

from oracle import oracle_sg, oracle_tc
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MODES = ["never", "auto", "always"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_17571_gb300 import wg
    c = wg.Context(0)
    yield c
    c.close()


def check(ctx, kind, g, **opts):
    cap = {"max_iters": opts["max_iters"]} if opts.get("max_iters") else {}
    want = (oracle_tc if kind == "tc" else oracle_sg)(g.src, g.dst, **cap)
    rel = ctx.load(g.src, g.dst)
    q = (ctx.tc if kind == "tc" else ctx.sg)(rel, **opts)
    from paper_2607_17571_gb300 import wg
    try:
        st = q.wait()
    except wg.WgError as e:
        assert e.code == wg.WG_E_ITER_CAP and opts.get("max_iters")
        st = q.poll()
    keys = q.result() if st.state != wg.WG_FAILED else None
    log = q.delta_sizes()
    q.free()
    rel.free()
    if keys is not None:  # a capped run reports its size, not its tuples
        assert keys.shape == want.keys.shape
        assert np.array_equal(keys, want.keys)
    assert st.n_tuples == want.keys.shape[0]
    assert st.iterations == want.iters
    assert log == want.log.tolist()
    return st


@pytest.mark.parametrize("mode", MODES)
def test_tc_graphs(ctx, mode):
    # long paths keep the candidates few for hundreds of iterations (the side
    # run fills and is folded back many times); ER and R-MAT closures shrink
    # their candidates late; a cycle derives its diagonal last
    for g in (I.path(300), I.er_graph(1000, 3000, 1), I.rmat_dag(12, 9000, 41), I.cycle(150),
              I.random_small(300, 900, 5)):
        check(ctx, "tc", g, side_run=mode)


@pytest.mark.parametrize("mode", MODES)
def test_sg_graphs(ctx, mode):
    for f in (I.sg_forest(3000, 6, 2.0, 0.01, 8), I.binary_tree(9)):
        check(ctx, "sg", f, side_run=mode)


@pytest.mark.parametrize("mode", ["auto", "always"])
def test_wide_keys(ctx, mode):
    # > 2^16 vertices: 17-bit ranks, 64-bit keys
    g = I.er_graph(70_000, 60_000, 29)
    check(ctx, "tc", g, side_run=mode)


@pytest.mark.parametrize("loop", [1, 2])  # WG_LOOP_HOST, WG_LOOP_HOST_STAGED
def test_host_loops(ctx, loop):
    for mode in ("auto", "always"):
        check(ctx, "tc", I.path(120), side_run=mode, loop=loop)
        check(ctx, "tc", I.er_graph(800, 2000, 3), side_run=mode, loop=loop)


@pytest.mark.parametrize("mode", ["auto", "always"])
def test_iteration_cap_mid_side_run(ctx, mode):
    # the cap ends the run in a side iteration: the result is both runs merged
    check(ctx, "tc", I.path(200), side_run=mode, max_iters=150)
    check(ctx, "tc", I.path(60), side_run=mode, max_iters=10)


def test_profiled_run(ctx):
    g = I.path(200)
    want = oracle_tc(g.src, g.dst)
    rel = ctx.load(g.src, g.dst)
    q = ctx.tc(rel, profile=True, side_run="always")
    q.wait()
    assert np.array_equal(q.result(), want.keys)
    prof = {p["name"]: p for p in q.profile()}
    assert prof["dedup_diff_merge"]["launches"] == want.iters + 1
    q.free()
    rel.free()


def test_regrowth_keeps_the_side_run():
    # a fresh context with minimal pools: the Full and side pools regrow
    # mid-run while the side run holds tuples (they must be carried over)
    from paper_2607_17571_gb300 import wg
    with wg.Context(0) as c:
        f = I.sg_forest(2189, 3, 2.0, 0.01, 1020)
        st = check(c, "sg", f, side_run="always", reserve_cand=1, reserve_full=1)
        assert st.regrows >= 2
        for g in (I.path(400), I.er_graph(900, 2700, 31), I.rmat_dag(11, 6000, 32)):
            check(c, "tc", g, side_run="always", reserve_cand=1, reserve_full=1)
            check(c, "tc", g, side_run="auto", reserve_cand=1, reserve_full=1)


def test_hash_join_and_full_width(ctx):
    g = I.rmat_dag(11, 6000, 33)
    for flags in (dict(hash_join=True), dict(full_width=True)):
        check(ctx, "tc", g, side_run="always", **flags)
        check(ctx, "tc", g, side_run="auto", **flags)


def test_engine_reuse_across_modes(ctx):
    # engines are cached per configuration: alternating modes on one
    # relation must not mix them up
    g = I.er_graph(1500, 4000, 17)
    want = oracle_tc(g.src, g.dst)
    rel = ctx.load(g.src, g.dst)
    for mode in ("always", "never", "auto", "always", "auto"):
        q = ctx.tc(rel, side_run=mode)
        q.wait()
        assert np.array_equal(q.result(), want.keys)
        assert q.delta_sizes() == want.log.tolist()
        q.free()
    rel.free()
