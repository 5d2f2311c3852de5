"""The generators reproduce, on this machine, the exact edge lists the stored
oracle results were computed from."""
import hashlib
import json
import os

import pytest

from paper_2607_17571_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))


@pytest.mark.parametrize("name", sorted(GOLD))
def test_workload_inputs_match_golden(name):
    g = I.workload(name)
    d = hashlib.sha256(g.src.astype("<u4").tobytes() + g.dst.astype("<u4").tobytes()).hexdigest()
    assert d == GOLD[name]["edges_sha256"]
    assert len(g) == GOLD[name]["n_edges"]


def test_golden_logs_are_consistent():
    for name, v in GOLD.items():
        assert sum(v["delta_sizes"]) == v["n_tuples"]          # disjoint deltas cover the closure
        assert v["delta_sizes"][-1] == 0 and len(v["delta_sizes"]) == v["iterations"] + 1
        assert all(x > 0 for x in v["delta_sizes"][1:-1])
