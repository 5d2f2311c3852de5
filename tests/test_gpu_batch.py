"""Batched and served fixpoints (wg_submit / wg_serve_step / wg_wait).

Every query's result must be byte-identical whether it runs alone (wg_tc /
wg_sg) or inside a mix of concurrent queries, and equal to the oracle;
queries submitted while others run join at the next iteration boundary;
when the pools cannot grow inside the memory budget the largest running
query is requeued and still finishes with the same result; a query that does
not fit even alone fails with WG_E_BUDGET.
"""
import functools

import numpy as np
import pytest

from oracle import oracle_sg, oracle_tc
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mix(seed, n_q=36):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_q):
        r = rng.random()
        if r < 0.55:
            n = int(np.exp(rng.uniform(np.log(16), np.log(900))))
            g = I.er_graph(n, int(n * rng.uniform(1.2, 2.5)), seed * 1000 + i)
            out.append(("tc", g))
        elif r < 0.8:
            g = I.sg_forest(int(rng.integers(50, 2500)), int(rng.integers(2, 9)), 2.0, 0.01,
                            seed * 1000 + i)
            out.append(("sg", g))
        else:
            g = I.rmat_dag(int(rng.integers(8, 12)), int(rng.integers(200, 3000)), seed * 1000 + i)
            out.append(("tc", g))
    return out


def _alone(ctx, kind, rel):
    q = (ctx.tc if kind == "tc" else ctx.sg)(rel)
    st = q.wait()
    res = (q.result(), q.delta_sizes(), st.iterations)
    q.free()
    return res


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_17571_gb300 import wg
    c = wg.Context(0)
    yield c
    c.close()


def test_alone_equals_mix_equals_oracle(ctx):
    from paper_2607_17571_gb300 import wg
    qs = _mix(1)
    rels = [ctx.load(g.src, g.dst) for _, g in qs]
    alone = [_alone(ctx, k, r) for (k, _), r in zip(qs, rels)]
    reqs = [(wg.WG_TC if k == "tc" else wg.WG_SG, r) for (k, _), r in zip(qs, rels)]
    handles = ctx.submit(reqs)
    for i, h in enumerate(handles):
        st = h.wait()
        assert st.state == wg.WG_DONE
        got = (h.result(), h.delta_sizes(), st.iterations)
        assert np.array_equal(got[0], alone[i][0]), i
        assert got[1] == alone[i][1] and got[2] == alone[i][2]
        h.free()
    for (k, g), a in list(zip(qs, alone))[::5]:
        want = (oracle_tc if k == "tc" else oracle_sg)(g.src, g.dst)
        assert np.array_equal(a[0], want.keys) and a[1] == want.log.tolist()
    for r in rels:
        r.free()


def test_continuous_admission(ctx):
    from paper_2607_17571_gb300 import wg
    qs = _mix(2, 30)
    rels = [ctx.load(g.src, g.dst) for _, g in qs]
    alone = [_alone(ctx, k, r) for (k, _), r in zip(qs, rels)]
    handles = []
    for wave in range(3):  # later waves arrive while earlier queries are on the GPU
        part = list(range(wave * 10, wave * 10 + 10))
        handles += ctx.submit([(wg.WG_TC if qs[i][0] == "tc" else wg.WG_SG, rels[i]) for i in part])
        ctx.serve_step(2)
    while ctx.serve_step(4) > 0:
        pass
    for i, h in enumerate(handles):
        st = h.poll()
        assert st.state == wg.WG_DONE
        assert np.array_equal(h.result(), alone[i][0]) and h.delta_sizes() == alone[i][1]
        h.free()
    for r in rels:
        r.free()


def test_slot_reuse_with_running_neighbours(ctx):
    # queries finish at very different times, so freed slots are reused while
    # their neighbours still run: only the new instances may be initialised
    from paper_2607_17571_gb300 import wg
    gs = [I.path(n) for n in (3, 40, 4, 60, 5, 35, 6, 50)] + [I.er_graph(300, 600, 9)] * 6
    want = [oracle_tc(g.src, g.dst) for g in gs]
    rels = [ctx.load(g.src, g.dst) for g in gs]
    hs = ctx.submit([(wg.WG_TC, r) for r in rels[:8]])
    for _ in range(3):
        ctx.serve_step(4)          # the short paths finish, their slots free up
    hs += ctx.submit([(wg.WG_TC, r) for r in rels[8:]])
    for h, w in zip(hs, want):
        h.wait()
        assert np.array_equal(h.result(), w.keys) and h.delta_sizes() == w.log.tolist()
        h.free()
    for r in rels:
        r.free()


def test_preemption_under_small_budget():
    from paper_2607_17571_gb300 import wg
    gs = [I.er_graph(n, 3 * n, 70 + n) for n in (300, 500, 700, 900, 1100, 1300)]
    want = [oracle_tc(g.src, g.dst) for g in gs]
    with wg.Context(0, mem_budget=320 << 20) as c:  # each fits alone, not all at once
        rels = [c.load(g.src, g.dst) for g in gs]
        hs = c.submit([(wg.WG_TC, r) for r in rels])
        for h, w in zip(hs, want):
            st = h.wait()
            assert st.state == wg.WG_DONE
            assert np.array_equal(h.result(), w.keys) and h.delta_sizes() == w.log.tolist()
            h.free()


def test_query_larger_than_budget_fails_cleanly():
    from paper_2607_17571_gb300 import wg
    g = I.er_graph(10000, 30000, 5)            # ~9e7 tuples: far beyond a 160 MB budget
    small = I.er_graph(200, 500, 6)
    with wg.Context(0, mem_budget=160 << 20) as c:
        big_rel, small_rel = c.load(g.src, g.dst), c.load(small.src, small.dst)
        hb, hs = c.submit([(wg.WG_TC, big_rel), (wg.WG_TC, small_rel)])
        with pytest.raises(wg.WgError) as e:
            hb.wait()
        assert e.value.code in (wg.WG_E_BUDGET, wg.WG_E_NOMEM)
        hs.wait()
        assert np.array_equal(hs.result(), oracle_tc(small.src, small.dst).keys)


def test_hopeless_large_request_fails_beside_small_ones():
    """A served request over 65,536 edges whose closure cannot fit the budget
    even alone fails with a budget error as soon as its growth is refused
    (it does not wait for the other engines to drain), and the small requests
    submitted around it complete with the oracle's results."""
    from paper_2607_17571_gb300 import wg
    big = I.er_graph(30000, 70000, 8)  # a giant component: ~5e8 tuples
    smalls = [I.er_graph(n, 3 * n, 500 + n) for n in (200, 400, 600, 800, 300, 700)]
    want = [oracle_tc(g.src, g.dst) for g in smalls]
    with wg.Context(0, mem_budget=256 << 20) as c:
        rb = c.load(big.src, big.dst)
        rs = [c.load(g.src, g.dst) for g in smalls]
        hs = c.submit([(wg.WG_TC, r) for r in rs[:3]] + [(wg.WG_TC, rb)] +
                      [(wg.WG_TC, r) for r in rs[3:]])
        with pytest.raises(wg.WgError) as e:
            hs[3].wait()
        assert e.value.code in (wg.WG_E_BUDGET, wg.WG_E_NOMEM)
        hs[3].free()
        for h, w in zip(hs[:3] + hs[4:], want):
            h.wait()
            assert np.array_equal(h.result(), w.keys) and h.delta_sizes() == w.log.tolist()
            h.free()


@functools.lru_cache(maxsize=1)
def _growth_cases():
    gs = [I.er_graph(n, 3 * n, 90 + n) for n in (800, 1400, 2000, 2600)]  # 0.6 .. 6.0 M tuples
    small = I.er_graph(300, 700, 17)
    return gs, [oracle_tc(g.src, g.dst) for g in gs], small, oracle_tc(small.src, small.dst)


@pytest.mark.parametrize("budget_mb", [72, 96, 128, 160, 200, 256, 320])
def test_failed_growth_leaves_engines_whole(budget_mb):
    """Pools that cannot grow within the budget, at whatever step of a growth
    the budget runs out (the candidate pools, the full-relation pools, the
    per-tile arrays, the retire pool): every query completes with the
    oracle's result or fails with a budget error, and later queries on the
    same context -- batched and alone, reusing the engines whose growth
    failed -- complete."""
    from paper_2607_17571_gb300 import wg
    gs, want, small, want_small = _growth_cases()
    with wg.Context(0, mem_budget=budget_mb << 20) as c:
        rels = [c.load(g.src, g.dst) for g in gs]
        srel = c.load(small.src, small.dst)
        for h, w in zip(c.submit([(wg.WG_TC, r) for r in rels]), want):
            try:
                h.wait()
                assert np.array_equal(h.result(), w.keys)
            except wg.WgError as e:
                assert e.code in (wg.WG_E_BUDGET, wg.WG_E_NOMEM)
            h.free()
        for r, w in [(srel, want_small)] + list(zip(rels[::-1], want[::-1])) + [(srel, want_small)]:
            q = None
            try:  # alone: the engine may not even get its first pools
                q = c.tc(r)
                q.wait()
                assert np.array_equal(q.result(), w.keys)
            except wg.WgError as e:
                assert e.code in (wg.WG_E_BUDGET, wg.WG_E_NOMEM)
            finally:
                if q is not None:
                    q.free()
        (h,) = c.submit([(wg.WG_TC, srel)])  # the batch engine's pools hold it
        h.wait()
        assert np.array_equal(h.result(), want_small.keys)
        h.free()


def _components(k, n, m, seed):
    """k disjoint ER graphs of n nodes and m edges each (vertex ids offset)."""
    gs = [I.er_graph(n, m, seed + i) for i in range(k)]
    src = np.concatenate([g.src + np.uint32(i * n) for i, g in enumerate(gs)]).astype(np.uint32)
    dst = np.concatenate([g.dst + np.uint32(i * n) for i, g in enumerate(gs)]).astype(np.uint32)
    return I.EdgeList(src, dst, dict(recipe=f"{k} x ER({n}, {m})"))


@functools.lru_cache(maxsize=2)
def _exclusive_cases(big_kind):
    if big_kind == "batch":  # > 4,096 vertices: its own batch engine; 6.3 M tuples
        big = I.er_graph(5000, 7000, 77)
    else:  # > 65,536 edges: served on a single-query engine; 9.9 M tuples
        big = _components(150, 500, 700, 900)
    smalls = [I.er_graph(n, 3 * n, 300 + n) for n in (800, 1100, 1400, 1700, 2000, 900, 1300, 1900)]
    return (big, smalls, oracle_tc(big.src, big.dst),
            [oracle_tc(g.src, g.dst) for g in smalls])


@pytest.mark.parametrize("big_kind", ["batch", "solo"])
@pytest.mark.parametrize("budget_mb", [96, 128, 192])
def test_query_that_fits_alone_completes_in_a_mix(budget_mb, big_kind):
    """A served request that completes when it is the only request finishes
    in a mix too, under the same budget with the same relations resident:
    when it cannot grow because other engines hold pools, it waits as the
    exclusive query for them to drain, then runs with the whole budget --
    in a batch engine, or (over 65,536 edges) on a single-query engine."""
    from paper_2607_17571_gb300 import wg
    big, smalls, want_big, want_smalls = _exclusive_cases(big_kind)

    def run(mix):
        with wg.Context(0, mem_budget=budget_mb << 20) as c:
            rb = c.load(big.src, big.dst)
            rs = [c.load(g.src, g.dst) for g in smalls]
            reqs = [(wg.WG_TC, r) for r in rs] if mix else []
            hs = c.submit(reqs[:4] + [(wg.WG_TC, rb)] + reqs[4:])
            wants = (want_smalls[:4] + [want_big] + want_smalls[4:]) if mix else [want_big]
            done = []
            for h, w in zip(hs, wants):
                try:
                    h.wait()
                    assert np.array_equal(h.result(), w.keys)
                    done.append(True)
                except wg.WgError as e:
                    assert e.code in (wg.WG_E_BUDGET, wg.WG_E_NOMEM)
                    done.append(False)
                h.free()
            return done[4] if mix else done[0]

    if run(mix=False):
        assert run(mix=True)


def test_large_requests_served_on_single_engines(ctx):
    """Served requests over 65,536 edges run one at a time on single-query
    engines beside the batch engines taking the small ones: every result
    equals the oracle's (and the per-iteration sizes too), whatever engine
    ran it."""
    from paper_2607_17571_gb300 import wg
    bigs = [_components(500, 100, 140, 900), _components(300, 200, 240, 1900)]
    smalls = [g for _, g in _mix(11, n_q=12)]
    gs = smalls[:6] + bigs[:1] + smalls[6:] + bigs[1:]
    kinds = [wg.WG_TC] * len(gs)
    want = [oracle_tc(g.src, g.dst) for g in gs]
    rels = [ctx.load(g.src, g.dst) for g in gs]
    hs = ctx.submit(list(zip(kinds, rels)))
    for h, w, g in zip(hs, want, gs):
        st = h.wait()
        assert np.array_equal(h.result(), w.keys) and h.delta_sizes() == w.log.tolist()
        if len(g) > (1 << 16):
            assert st.gpu_launches > 0  # launched by its own engine
        h.free()
    for r in rels:
        r.free()


def test_iteration_cap_in_batch(ctx):
    from paper_2607_17571_gb300 import wg
    g = I.path(40)
    rel = ctx.load(g.src, g.dst)
    h, h2 = ctx.submit([(wg.WG_TC, rel, dict(max_iters=7)), (wg.WG_TC, rel)])
    with pytest.raises(wg.WgError) as e:
        h.wait()
    assert e.value.code == wg.WG_E_ITER_CAP
    assert h.delta_sizes() == oracle_tc(g.src, g.dst, max_iters=7).log.tolist()
    h2.wait()
    assert h2.poll().iterations == 39
    h.free()
    h2.free()
    rel.free()
