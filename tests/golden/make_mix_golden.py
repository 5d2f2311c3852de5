"""Write the oracle results of the batched and served query mixes:

    tests/golden/batch4096.json   every query of the 4,096-query batch mix
    tests/golden/serve_pool.json  every request of the served mix's pool

Calls only oracle/ (and the seeded generators for the inputs).  Per query:
kind, edge count, closure size, iteration count and the digest of the sorted
result (oracle.digest_keys: the sum wg_result_digest computes on the device),
so the benchmarks can check every result without copying it.  TC queries use
the reachability form of the oracle (oracle_tc_reach), SG queries the
semi-naive oracle_sg.  Small queries run in a process pool (spawn), large ones
one at a time with every host thread.

    python tests/golden/make_mix_golden.py [--batch N] [--pool N] [--only batch|serve]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

HERE = os.path.dirname(os.path.abspath(__file__))
BIG_EDGES = 60_000  # TC queries above this run alone with every thread


def _solve(job):
    kind, idx, threads = job
    from oracle import digest_keys, oracle_sg, oracle_tc_reach
    from paper_2607_17571_gb300 import inputs as I
    if kind == "batch":
        n, m, s = I.batch_query_sizes(idx + 1)[idx]
        qk, g = "tc", I.er_graph(n, m, s)
    else:
        qk, g = I.serve_request(idx)
    if qk == "tc":
        cnt, iters, _, dg = oracle_tc_reach(g.src, g.dst, n_threads=threads)
    else:
        r = oracle_sg(g.src, g.dst)
        cnt, iters, dg = int(r.keys.shape[0]), int(r.iters), digest_keys(r.keys)
    return idx, dict(kind=qk, n_edges=len(g), n_tuples=int(cnt), iterations=int(iters),
                     digest=str(dg))


def _sizes(kind, count):
    from paper_2607_17571_gb300 import inputs as I
    if kind == "batch":
        return [m for (_, m, _) in I.batch_query_sizes(count)]
    return [len(I.serve_request(r)[1]) for r in range(count)]


def run(kind, count, out):
    t = time.time()
    sizes = _sizes(kind, count)
    small = [i for i in range(count) if sizes[i] <= BIG_EDGES]
    big = [i for i in range(count) if sizes[i] > BIG_EDGES]
    res = {}
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for i, r in pool.imap_unordered(_solve, [(kind, i, 1) for i in small], chunksize=4):
            res[i] = r
    for i in big:
        res[i] = _solve((kind, i, os.cpu_count()))[1]
        print(kind, i, res[i], flush=True)
    data = {"count": count, "oracle_seconds": round(time.time() - t, 1),
            "oracle_threads": os.cpu_count(),
            "queries": [res[i] for i in range(count)]}
    with open(out, "w") as f:
        json.dump(data, f, separators=(",", ":"))
    print(kind, "done", count, "queries", data["oracle_seconds"], "s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--pool", type=int, default=500)
    ap.add_argument("--only", default=None, choices=["batch", "serve"])
    a = ap.parse_args()
    if a.only in (None, "batch"):
        run("batch", a.batch, os.path.join(HERE, "batch4096.json"))
    if a.only in (None, "serve"):
        run("serve", a.pool, os.path.join(HERE, "serve_pool.json"))


if __name__ == "__main__":
    main()
