"""Failure detection without a GPU fault: a bounded device wait that runs
out.  One warp runs the decoupled-lookback wait of the scan stages on a
predecessor whose status word nothing ever publishes; the wait gives up after
its poll limit, the kernel records the timeout and returns, the host reports
WG_E_DEVICE_TIMEOUT, and the same context then computes a fixpoint that
equals the oracle's."""
import numpy as np
import pytest

from oracle import oracle_tc
from paper_2607_17571_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_stays_usable():
    from paper_2607_17571_gb300 import wg
    with wg.Context(0) as c:
        assert c.selftest_wait_timeout() == wg.WG_E_DEVICE_TIMEOUT
        g = I.er_graph(400, 1000, 8)
        q = c.tc(c.load(g.src, g.dst))
        q.wait()
        want = oracle_tc(g.src, g.dst)
        assert np.array_equal(q.result(), want.keys) and q.delta_sizes() == want.log.tolist()
        q.free()
        # the context's sort primitive still sorts (its control block starts clear)
        import torch
        keys = np.random.default_rng(3).integers(0, 2 ** 32, 200_000, dtype=np.uint64).astype(np.uint32)
        t = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        torch.cuda.synchronize()
        c.sort_keys(t.data_ptr(), keys.shape[0], 4, 32)
        assert np.array_equal(t.cpu().numpy().view(np.uint32), np.sort(keys))
