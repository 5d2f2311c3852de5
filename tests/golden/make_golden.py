"""Write tests/golden/workloads.json: oracle results of the full-size workloads.

Calls only oracle/ (and the seeded generators for the inputs).  For each
workload it stores the digest of the generated edge list (so a test can tell
that the inputs on another machine are the same), the closure size, the
SHA-256 of the sorted packed keys (little-endian uint64), the iteration count
and the per-iteration delta sizes.

The R-MAT TC closures (478,120,144 tuples on 2^17 nodes) are computed row by row with
oracle_tc_rows over every source (exact: the TC rule never changes the first
component), using all host cores.

    python tests/golden/make_golden.py [--only NAME]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import digest_keys, oracle_sg, oracle_tc, oracle_tc_reach, oracle_tc_rows  # noqa: E402
from paper_2607_17571_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")


def edge_digest(g):
    return hashlib.sha256(g.src.astype("<u4").tobytes() + g.dst.astype("<u4").tobytes()).hexdigest()


def key_digest(keys):
    return hashlib.sha256(np.ascontiguousarray(keys, dtype="<u8").tobytes()).hexdigest()


def run(name):
    g = I.workload(name)
    t = time.time()
    if name.startswith("sg_"):
        r = oracle_sg(g.src, g.dst)
        keys, log, iters = r.keys, r.log.tolist(), r.iters
    elif name.startswith("tc_rmat"):
        srcs = np.unique(g.src)
        keys, _, log_sum, mx = oracle_tc_rows(g.src, g.dst, srcs, n_threads=os.cpu_count())
        iters = max(1, mx)
        log = log_sum[: iters + 1].tolist()
    else:
        r = oracle_tc(g.src, g.dst)
        keys, log, iters = r.keys, r.log.tolist(), r.iters
    dt = time.time() - t
    out = dict(edges_sha256=edge_digest(g), n_edges=len(g), n_tuples=int(keys.shape[0]),
               keys_sha256=key_digest(keys), keys_digest=str(digest_keys(keys)),
               iterations=int(iters), delta_sizes=[int(x) for x in log],
               oracle_seconds=round(dt, 1), oracle_threads=os.cpu_count())
    if name.startswith("tc_"):
        # the reachability form of the oracle must agree on every figure
        n, it, lg, dg = oracle_tc_reach(g.src, g.dst, n_threads=os.cpu_count())
        assert (n, it, lg.tolist(), str(dg)) == (out["n_tuples"], out["iterations"],
                                                 out["delta_sizes"], out["keys_digest"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in ("tc_er_1k", "sg_forest_60k", "tc_rmat17_400k", "tc_rmat19_400k"):
        if a.only and name != a.only:
            continue
        data[name] = run(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
