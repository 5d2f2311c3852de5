"""Tile shapes of the join count and of the fused deduplication / set
difference / merge pass, the radix-sort modes of single TC queries, and the
autotuner that picks them (wg_autotune, wg_set_tiles, wg_set_sort).

Every compiled shape must give the oracle's result bit for bit -- closure,
iteration count and per-iteration delta sizes -- for TC and SG, single and
batched queries, 32-bit and 64-bit keys, on graphs that span many tiles of
either shape with a ragged last tile.  The autotuner must choose among the
compiled candidates and engines created afterwards must use its choice.
"""
import functools

import numpy as np
import pytest

from oracle import oracle_sg, oracle_tc
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COUNT = (2048, 1024)
FUSE = {4: (4096, 2048), 8: (2048, 1024)}
EMIT = (4096, 2048)


def _components(k, n, m, seed):
    """k disjoint ER graphs of n nodes and m edges each (vertex ids offset)."""
    gs = [I.er_graph(n, m, seed + i) for i in range(k)]
    src = np.concatenate([g.src + np.uint32(i * n) for i, g in enumerate(gs)]).astype(np.uint32)
    dst = np.concatenate([g.dst + np.uint32(i * n) for i, g in enumerate(gs)]).astype(np.uint32)
    return I.EdgeList(src, dst, dict(recipe=f"{k} x ER({n}, {m})"))


@functools.lru_cache(maxsize=1)
def _cases():
    tc32 = I.rmat_dag(12, 12_000, 41)                  # 32-bit keys, many tiles per iteration
    sg32 = I.sg_forest(3000, 4, 2.0, 0.01, 42)
    tc64 = _components(700, 100, 140, 43)             # 70,000 vertices: 64-bit keys
    smalls = [I.er_graph(n, 2 * n, 50 + n) for n in (90, 300, 700, 1500)]
    return dict(
        tc32=(tc32, oracle_tc(tc32.src, tc32.dst)),
        sg32=(sg32, oracle_sg(sg32.src, sg32.dst)),
        tc64=(tc64, oracle_tc(tc64.src, tc64.dst)),
        smalls=[(g, oracle_tc(g.src, g.dst)) for g in smalls],
    )


def _check(q, want):
    q.wait()
    assert np.array_equal(q.result(), want.keys)
    assert q.delta_sizes() == want.log.tolist()
    q.free()


@pytest.mark.parametrize("count_tile", COUNT)
@pytest.mark.parametrize("half_fuse", [False, True])
@pytest.mark.parametrize("emit_tile", EMIT)
def test_every_tile_shape_matches_oracle(count_tile, half_fuse, emit_tile):
    from paper_2607_17571_gb300 import wg
    cases = _cases()
    with wg.Context(0) as c:
        for kb in (4, 8):
            c.set_tiles(kb, count_tile, FUSE[kb][1 if half_fuse else 0], emit_tile)
        g, want = cases["tc32"]
        rel = c.load(g.src, g.dst)
        _check(c.tc(rel), want)
        _check(c.tc(rel, loop=wg.WG_LOOP_HOST), want)
        _check(c.tc(rel, full_width=True), want)
        g, want = cases["sg32"]
        _check(c.sg(c.load(g.src, g.dst)), want)
        g, want = cases["tc64"]
        rel64 = c.load(g.src, g.dst)
        assert rel64.info()["field_bits"] > 16
        _check(c.tc(rel64), want)
        rels = [c.load(g.src, g.dst) for g, _ in cases["smalls"]]
        hs = c.submit([(wg.WG_TC, r) for r in rels])
        for h, (_, want) in zip(hs, cases["smalls"]):
            _check(h, want)


def _hub():
    # source 0 -> 1..1000, each of them -> 1001..1600: in its first iteration
    # source 0 has 600,000 candidates (147 tiles), more than the per-segment
    # sort takes, so its launches fall back to the lookback passes (with
    # 9-bit digits the per-segment sort takes it all the same)
    mid = np.arange(1, 1001, dtype=np.uint32)
    leaf = np.arange(1001, 1601, dtype=np.uint32)
    src = np.concatenate([np.zeros(1000, np.uint32), np.repeat(mid, 600)])
    dst = np.concatenate([mid, np.tile(leaf, 1000)])
    return I.EdgeList(src, dst, dict(recipe="hub"))


# WG_SORT_SEGMENT16, WG_SORT_SEGMENT8, WG_SORT_PASSES, WG_SORT_SEGMENT_WIDE
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_every_sort_mode_matches_oracle(mode):
    from paper_2607_17571_gb300 import wg
    cases = _cases()
    hub = _hub()
    want_hub = oracle_tc(hub.src, hub.dst)
    with wg.Context(0) as c:
        for kb in (4, 8):
            c.set_sort(kb, mode)
        for name in ("tc32", "tc64"):
            g, want = cases[name]
            rel = c.load(g.src, g.dst)
            _check(c.tc(rel), want)
            _check(c.tc(rel, loop=wg.WG_LOOP_HOST, profile=True), want)
        _check(c.tc(c.load(hub.src, hub.dst)), want_hub)
    with wg.Context(0) as c, pytest.raises(wg.WgError):
        c.set_sort(4, 4)


# 8, 9, 15, 17 and 18-bit fields (mean degree 0.9: small closures)
@pytest.mark.parametrize("n", [150, 300, 20_000, 100_000, 200_000])
def test_wide_digit_sort_field_widths(n):
    """The per-segment sort with digits of up to 9 bits: one pass for fields
    of at most 8 bits, two passes of ceil(w/2) bits for 9..18-bit fields
    (17 and 18 bits: two passes instead of three)."""
    from paper_2607_17571_gb300 import wg
    g = I.er_graph(n, int(n * 0.9), 300 + n % 97)
    want = oracle_tc(g.src, g.dst)
    with wg.Context(0) as c:
        c.set_sort(4, wg.WG_SORT_SEGMENT_WIDE)
        c.set_sort(8, wg.WG_SORT_SEGMENT_WIDE)
        rel = c.load(g.src, g.dst)
        _check(c.tc(rel), want)
        _check(c.tc(rel, side_run="never"), want)


def test_autotune_picks_a_compiled_shape_and_engines_use_it():
    from paper_2607_17571_gb300 import wg
    g, want = _cases()["tc32"]
    with wg.Context(0) as c:
        rel = c.load(g.src, g.dst)
        t = c.autotune(rel, wg.WG_TC)
        assert t["key_bytes"] == 4
        assert t["count_cand"] == list(COUNT) and t["fuse_cand"] == list(FUSE[4])
        assert t["emit_cand"] == list(EMIT)
        assert t["count_tile"] in COUNT and t["fuse_tile"] in FUSE[4] and t["emit_tile"] in EMIT
        assert all(ms > 0 for ms in t["count_ms"] + t["fuse_ms"] + t["emit_ms"])
        # the choice is the faster candidate of each stage
        assert t["count_tile"] == COUNT[int(t["count_ms"][1] < t["count_ms"][0])]
        assert t["fuse_tile"] == FUSE[4][int(t["fuse_ms"][1] < t["fuse_ms"][0])]
        assert t["emit_tile"] == EMIT[int(t["emit_ms"][1] < t["emit_ms"][0])]
        # the radix sort of the per-source segments: the fastest of the four modes
        assert all(ms > 0 for ms in t["sort_ms"])
        assert t["sort_mode"] == int(np.argmin(t["sort_ms"]))
        _check(c.tc(rel), want)
        h, = c.submit([(wg.WG_TC, rel)])
        _check(h, want)


def test_set_tiles_rejects_shapes_that_are_not_compiled():
    from paper_2607_17571_gb300 import wg
    with wg.Context(0) as c:
        for args in ((4, 3000, 0), (4, 0, 1000), (8, 0, 4096), (2, 0, 0), (4, 0, 0, 1024)):
            with pytest.raises(wg.WgError) as e:
                c.set_tiles(*args)
            assert e.value.code == wg.WG_E_INVAL
        c.set_tiles(4, 0, 0)  # back to the defaults
