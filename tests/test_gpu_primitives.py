"""Each sorted-array stage alone, through the C-ABI, against plain library
routines on the host: radix sort vs np.sort, fused dedup + set difference vs
np.unique + np.setdiff1d, disjoint merge vs np.sort of the concatenation.
Sizes straddle the 4096-key tile (0, 1, tile - 1, tile, tile + 1, many tiles
with a ragged tail); keys include 0 and the all-ones maximum."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_17571_gb300 import wg
    c = wg.Context(0)
    yield c
    c.close()


def _dev(a):
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.int32 if a.dtype == np.uint32 else np.int64).copy()).cuda()
    return t


def _host(t, dtype):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(dtype)


def _keys(rng, n, kb, bits):
    dt = np.uint32 if kb == 4 else np.uint64
    v = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).astype(np.uint64)
    if bits < 64:
        v &= np.uint64((1 << bits) - 1)
    v = v.astype(dt)
    if n > 2:
        v[0] = 0
        v[1] = dt((1 << bits) - 1) if bits < 64 else np.iinfo(dt).max
    return v


@pytest.mark.parametrize("kb,bits", [(4, 8), (4, 20), (4, 32), (8, 34), (8, 48), (8, 64)])
@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 100_003, 2_500_001])
def test_sort(ctx, kb, bits, n):
    if bits > 8 * kb:
        pytest.skip()
    rng = np.random.default_rng(n * 131 + bits)
    a = _keys(rng, n, kb, bits)
    t = _dev(a) if n else torch.zeros(1, dtype=torch.int32 if kb == 4 else torch.int64, device="cuda")
    ctx.sort_keys(t.data_ptr(), n, kb, bits)
    got = _host(t, a.dtype)[:n]
    assert np.array_equal(got, np.sort(a))


def test_sort_clustered_and_equal_keys(ctx):
    # long runs of equal high digits (as in grouped join output) and all-equal keys
    a = np.repeat(np.arange(50, dtype=np.uint32) << 16, 3000) | np.tile(
        np.arange(3000, dtype=np.uint32)[::-1], 50)
    t = _dev(a)
    ctx.sort_keys(t.data_ptr(), a.shape[0], 4, 32)
    assert np.array_equal(_host(t, np.uint32), np.sort(a))
    b = np.full(100_000, 12345, dtype=np.uint64)
    t = _dev(b)
    ctx.sort_keys(t.data_ptr(), b.shape[0], 8, 40)
    assert np.array_equal(_host(t, np.uint64), b)


@pytest.mark.parametrize("kb", [4, 8])
@pytest.mark.parametrize("n,nf", [(1, 0), (1, 1), (5000, 0), (4096, 100), (30000, 2000),
                                  (200_001, 1_000_000), (1_000_000, 50)])
def test_unique_diff(ctx, kb, n, nf):
    dt = np.uint32 if kb == 4 else np.uint64
    rng = np.random.default_rng(n + nf)
    hi = max(4, n // 3)
    cand = np.sort(rng.integers(0, hi, size=n).astype(dt))
    full = np.unique(rng.integers(0, hi, size=nf).astype(dt)) if nf else np.zeros(0, dt)
    tc, tf = _dev(cand), _dev(full) if full.shape[0] else None
    out = torch.empty_like(tc)
    m = ctx.unique_diff(tc.data_ptr(), n, tf.data_ptr() if tf is not None else 0, full.shape[0],
                        out.data_ptr(), kb)
    want = np.setdiff1d(np.unique(cand), full)
    got = _host(out, dt)[:m]
    assert m == want.shape[0] and np.array_equal(got, want)


@pytest.mark.parametrize("kb", [4, 8])
@pytest.mark.parametrize("na,nb", [(0, 5), (5, 0), (1, 1), (4096, 1), (10_000, 10_000),
                                   (1_000_003, 77), (3, 500_000)])
def test_merge_disjoint(ctx, kb, na, nb):
    dt = np.uint32 if kb == 4 else np.uint64
    rng = np.random.default_rng(na * 7 + nb)
    u = np.unique(rng.integers(0, 4 * (na + nb) + 10, size=2 * (na + nb) + 10).astype(dt))
    rng.shuffle(u)
    a, b = np.sort(u[:na]), np.sort(u[na:na + nb])
    ta = _dev(a) if na else None
    tb = _dev(b) if nb else None
    out = torch.empty(max(1, na + nb), dtype=torch.int32 if kb == 4 else torch.int64, device="cuda")
    ctx.merge_disjoint(ta.data_ptr() if ta is not None else 0, na,
                       tb.data_ptr() if tb is not None else 0, nb, out.data_ptr(), kb)
    assert np.array_equal(_host(out, dt)[: na + nb], np.sort(np.concatenate([a, b])))
