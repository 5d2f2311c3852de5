"""wg_sort_keys_noalloc: the radix sort for callers that cannot allocate
device memory (code inside another runtime's memory arena, or a process that
must keep its device footprint fixed).  It takes only the caller's key buffer
and a stream; its scratch is a static device array inside the library.

Checked through the C-ABI against the context-based wg_sort_keys, bit for bit
(integer keys: exact equality), on two calls in a row so that the second call
runs on the scratch the first one left behind; on a non-default stream; a size
above the stated maximum must be refused without touching the keys; and a
bounded device wait that gives up must be reported by the next check (a call
with n = 0).  This file is collected last so that a failure here never hides
the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _random_keys(rng, n, kb, bits):
    v = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).astype(np.uint64)
    v &= np.uint64((1 << bits) - 1)
    return v.astype(np.uint32 if kb == 4 else np.uint64)


def _to_dev(a):
    return torch.from_numpy(a.view(np.int32 if a.dtype == np.uint32 else np.int64).copy()).cuda()


def test_noalloc_sort_matches_wg_sort_keys_on_two_calls():
    from paper_2607_17571_gb300 import wg
    rng = np.random.default_rng(2024)
    cases = [(4, 32, 700_001), (8, 40, wg.WG_NOALLOC_MAX_KEYS)]  # the second call is the largest
    with wg.Context(0) as ctx:
        for kb, bits, n in cases:
            keys = _random_keys(rng, n, kb, bits)
            ref = _to_dev(keys)
            ctx.sort_keys(ref.data_ptr(), n, kb, bits)          # the existing entry point
            got = _to_dev(keys)
            torch.cuda.synchronize()
            wg.sort_keys_noalloc(got.data_ptr(), n, kb, bits)   # legacy default stream
            torch.cuda.synchronize()
            assert torch.equal(got, ref)
            assert np.array_equal(got.cpu().numpy().view(keys.dtype), np.sort(keys))


def test_noalloc_sort_on_a_non_default_stream():
    """Keys produced on a torch stream and sorted on it (odd pass count: 40-bit
    keys take five 8-bit passes and a copy back); only that stream is
    synchronised before the result is read."""
    from paper_2607_17571_gb300 import wg
    rng = np.random.default_rng(77)
    s = torch.cuda.Stream()
    for kb, bits, n in [(8, 40, 333_333), (4, 24, 65_537)]:
        keys = _random_keys(rng, n, kb, bits)
        host = torch.from_numpy(keys.view(np.int32 if kb == 4 else np.int64).copy()).pin_memory()
        with torch.cuda.stream(s):
            t = torch.empty_like(host, device="cuda")
            t.copy_(host, non_blocking=True)      # produced on s
            wg.sort_keys_noalloc(t.data_ptr(), n, kb, bits, s.cuda_stream)
            out = t.to("cpu", non_blocking=False)
        s.synchronize()
        assert np.array_equal(out.numpy().view(keys.dtype), np.sort(keys))


def test_noalloc_sort_refuses_sizes_above_the_maximum():
    from paper_2607_17571_gb300 import wg
    n = wg.WG_NOALLOC_MAX_KEYS + 1
    keys = np.arange(n, dtype=np.uint32)[::-1].copy()
    t = _to_dev(keys)
    torch.cuda.synchronize()
    with pytest.raises(wg.WgError) as e:
        wg.sort_keys_noalloc(t.data_ptr(), n, 4, 32)
    assert e.value.code == wg.WG_E_CAPACITY
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().view(np.uint32), keys)


def test_noalloc_wait_timeout_is_reported_by_the_next_check():
    """Failure detection without a GPU fault: the self-test runs the lookback
    wait in the scratch's control block on a status word nothing publishes;
    the wait gives up and records it.  The next check reports
    WG_E_DEVICE_TIMEOUT and clears the record, the one after reports WG_OK,
    and a sort afterwards is correct."""
    from paper_2607_17571_gb300 import wg
    wg.noalloc_check()  # start from a clear record (earlier tests may have left one)
    with wg.Context(0) as ctx:
        assert ctx.selftest_wait_timeout() == wg.WG_E_DEVICE_TIMEOUT
    assert wg.noalloc_check() == wg.WG_E_DEVICE_TIMEOUT
    assert wg.noalloc_check() == wg.WG_OK
    rng = np.random.default_rng(5)
    keys = _random_keys(rng, 100_000, 4, 32)
    t = _to_dev(keys)
    torch.cuda.synchronize()
    wg.sort_keys_noalloc(t.data_ptr(), keys.shape[0], 4, 32)
    assert wg.noalloc_check() == wg.WG_OK
    assert np.array_equal(t.cpu().numpy().view(np.uint32), np.sort(keys))
