"""The N > 1 path of bench.py (replicas: one independent fixpoint per rank,
no collective on the data path) reduces over ranks exactly as its contract
says: the whole-job value is all ranks' tuples over the SLOWEST rank's time.
Two gloo ranks on the CPU, rendezvous on 127.0.0.1."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)  # WORLD_SIZE, RANK, LOCAL_RANK
        tuples = 1000 * (rank + 1)          # each replica's closure size
        ms = 50.0 + 25.0 * rank             # each replica's timed region
        tot, mx = bench.aggregate(tuples, ms)
        mins = bench.combine_ranks([ms], dist.ReduceOp.MIN)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"tot": tot, "max_ms": mx, "min_ms": mins[0]}, f)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["tot"] == 3000.0          # 1000 + 2000 tuples
        assert d["max_ms"] == 75.0         # the slowest rank's time
        assert d["min_ms"] == 50.0
    # the bench's whole-job value for these ranks
    assert 3000.0 / (75.0 / 1e3) == pytest.approx(40000.0)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1234, 5.0) == (1234.0, 5.0)
    assert bench.combine_ranks([1.0, 2.0], None) == [1.0, 2.0]
