"""The round-trip that __graft_entry__.smoke() performs (one TC and one SG
fixpoint on cuda:0 checked against the oracle) stays runnable."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import __graft_entry__
    __graft_entry__.smoke()
