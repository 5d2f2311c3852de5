#!/usr/bin/env python3
"""Benchmark of the semi-naive fixpoint on one or more GPUs.

A step is one complete fixpoint (every iteration of join, radix sort, fused
dedup + set difference and merge, with the loop on the device) of the
workload over a relation already resident in device memory.  Default
workload: transitive closure of an R-MAT(0.57, 0.19, 0.19, 0.05) graph with
2^17 nodes and 400k distinct DAG edges (random relabel, src < dst kept), seed 2
-- 478,120,144 closure tuples in 15 iterations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload tc_rmat17_400k|sg_forest_60k|tc_er_1k]

Multi-GPU (torchrun, one rank per GPU): the path is run as independent
replicas (each rank computes the whole fixpoint; no collective on the data
path); value = tuples of all ranks / max-over-ranks time ("weak" scaling).
`--impl reference` times the CPU oracle (tests' semi-naive std::set
evaluator, row by row over all host cores) on a bounded sample of sources.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fixpoint derived tuples/s"
UNIT = "tuples/s"
WORKLOADS = {
    "tc_rmat17_400k": dict(kind="tc", desc="TC, R-MAT(.57,.19,.19,.05) 2^17 nodes, 400k distinct "
                                            "DAG edges (random relabel, src<dst), seed 2"),
    "sg_forest_60k": dict(kind="sg", desc="SG, forest of 60k nodes (40 roots, Poisson(2) "
                                          "branching) + 1% equal-depth cross edges, seed 3"),
    "tc_er_1k": dict(kind="tc", desc="TC, directed Erdos-Renyi 1,000 nodes, 3,000 edges, seed 1"),
    "tc_rmat15_100k": dict(kind="tc", desc="TC, R-MAT(.57,.19,.19,.05) 2^15 nodes, 100k distinct "
                                           "DAG edges, seed 2 (profiling-size case)"),
    "tc_rmat19_400k": dict(kind="tc", desc="TC, R-MAT(.57,.19,.19,.05) 2^19 nodes, 400k distinct "
                                           "DAG edges, seed 2 (124,568 vertices: 17-bit ranks, "
                                           "64-bit keys)"),
    "tc_rmat19_150k": dict(kind="tc", desc="TC, R-MAT(.57,.19,.19,.05) 2^19 nodes, 150k distinct "
                                           "DAG edges, seed 2 (76,647 vertices: 64-bit keys; "
                                           "profiling-size case)"),
}
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def combine_ranks(values, reduce_op):
    """All-reduce helper over torch.distributed (identity when world == 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return values
    t = torch.tensor(values, dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=reduce_op)
    return t.cpu().tolist()


def aggregate(per_rank_tuples, per_rank_ms):
    """Whole-job throughput: all tuples over the slowest rank's time."""
    import torch.distributed as dist
    tot = combine_ranks([float(per_rank_tuples)], dist.ReduceOp.SUM)[0]
    mx = combine_ranks([float(per_rank_ms)], dist.ReduceOp.MAX)[0]
    return tot, mx


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(g, kind, budget_s, seed=0, threads=None):
    """The oracle as it stands on the host cores, on a bounded sample."""
    import oracle
    threads = threads or os.cpu_count()
    rng = np.random.default_rng(seed)
    if kind == "tc":
        srcs = rng.permutation(np.unique(g.src))
        take = 64
        done_tuples, done_s, n_src = 0, 0.0, 0
        while done_s < budget_s and n_src < srcs.shape[0]:
            sample = np.sort(srcs[n_src:n_src + take])
            t = time.perf_counter()
            keys, _, _, _ = oracle.oracle_tc_rows(g.src, g.dst, sample, n_threads=threads)
            done_s += time.perf_counter() - t
            done_tuples += keys.shape[0]
            n_src += sample.shape[0]
            take *= 2
        return dict(value=done_tuples / done_s, unit=UNIT, cores=threads, kind="oracle",
                    sample=f"rows T(x,.) of {n_src} random sources of {srcs.shape[0]} "
                           f"({done_tuples} tuples, {done_s:.1f} s)", seconds=done_s)
    # SG does not split by rows: run the whole oracle with a wall-clock budget note
    t = time.perf_counter()
    r = oracle.oracle_sg(g.src, g.dst)
    dt = time.perf_counter() - t
    return dict(value=r.keys.shape[0] / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"whole fixpoint ({r.keys.shape[0]} tuples, {dt:.1f} s)", seconds=dt)


def run_reference(args):
    from paper_2607_17571_gb300 import inputs as I
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    g = I.workload(args.workload)
    threads = os.cpu_count()
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(g, wl["kind"], args.ref_step_seconds, seed=k, threads=threads)
        if k >= args.warmup:
            vals.append(cb)
    v = statistics.mean(c["value"] for c in vals)
    # each step is a bounded sample of the workload, not the whole fixpoint:
    # ms_per_step is the sample's timed seconds, and "note" says which oracle ran
    ms = 1e3 * statistics.mean(c["seconds"] for c in vals)
    note = ("row-wise TC oracle (reachability rows of random sources) on a sample; "
            "throughput of that sample, not of the semi-naive fixpoint"
            if wl["kind"] == "tc" else "whole semi-naive SG oracle, one thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak",
            "note": note,
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2607_17571_gb300 import inputs as I
    from paper_2607_17571_gb300 import wg

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    g = I.workload(args.workload)
    n = len(g)
    ctx = wg.Context(local)
    stream = ctx.torch_stream
    src_t = torch.from_numpy(g.src.view(np.int32)).cuda(local)
    dst_t = torch.from_numpy(g.dst.view(np.int32)).cuda(local)
    torch.cuda.synchronize()
    rel = ctx.load_device(src_t.data_ptr(), dst_t.data_ptr(), n)
    info = rel.info()
    run0 = ctx.tc if wl["kind"] == "tc" else ctx.sg
    loop = {"host": wg.WG_LOOP_HOST, "staged": wg.WG_LOOP_HOST_STAGED}.get(args.loop,
                                                                          wg.WG_LOOP_DEVICE)

    def run(r, **kw):
        return run0(r, loop=loop, **kw)
    kb = 4 if 2 * info["field_bits"] <= 32 else 8
    tiles = None if args.no_autotune else autotune_ctx(
        ctx, [rel], wg.WG_TC if wl["kind"] == "tc" else wg.WG_SG)

    # warm-up: also sizes the pools (a relation remembers the capacities it needed)
    st = None
    for _ in range(args.warmup):
        q = run(rel)
        st = q.wait()
        q.free()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > L2 (129 MB)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms, tuples, launches, iters, regrows = [], 0, 0, 0, 0
    torch.cuda.nvtx.range_push("wg_timed")  # lets a profiler select the timed steps
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)                     # evict L2 between steps (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q = run(rel)
        st = q.wait()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        tuples += st.n_tuples
        launches += st.gpu_launches
        iters, regrows = st.iterations, regrows + st.regrows
        q.free()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(ms)
    all_tuples, max_ms = aggregate(tuples, total_ms)
    value = all_tuples / (max_ms / 1e3)

    # roofline: the same fixpoint once more with CUDA events around every kernel
    q = run(rel, profile=True)
    q.wait()
    prof = q.profile()
    q.free()
    dom = max(prof, key=lambda p: p["total_ms"])
    peak, peak_src = read_peaks()
    per_launch_bytes = dom["bytes"] / dom["launches"]
    per_launch_ms = dom["total_ms"] / dom["launches"]
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if os.path.exists(tfile):
        for line in open(tfile):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == args.workload and parts[1] == dom["name"]:
                traffic = float(parts[2])
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom["name"],
            "frac_of_nominal_7900": round(achieved / 7900.0, 4),  # nominal HBM3e, context
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
            else "fallback 6.8 TB/s",
            "per_kernel": [{"name": p["name"], "launches": p["launches"],
                            "ms": round(p["total_ms"], 3),
                            "GBps": round(p["bytes"] / (p["total_ms"] / 1e3) / 1e9, 1),
                            "share": round(p["total_ms"] / sum(x["total_ms"] for x in prof), 4)}
                           for p in sorted(prof, key=lambda p: -p["total_ms"])]}

    # end to end through the public C-ABI with host buffers: H2D of the edge
    # list, the fixpoint, D2H of the sorted result
    e2e_ms, h2d, d2h = [], 2 * 4 * n, 0
    if args.e2e_steps:
        # page-locked host buffers, allocated once like a server's I/O buffers:
        # the edge list the user uploads and the result they read back
        src_h, dst_h = wg.pinned(n, np.uint32), wg.pinned(n, np.uint32)
        src_h[:], dst_h[:] = g.src, g.dst
        res_h = wg.pinned(st.n_tuples)
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r2 = ctx.load(src_h, dst_h)
        q = run(r2)
        q.wait()
        res = q.result(out=res_h)
        e2e_ms.append((time.perf_counter() - t) * 1e3)
        d2h = res.nbytes
        q.free()
        r2.free()
        del res
    e2e = None
    if e2e_ms:
        e2e_tuples, e2e_max = aggregate(st.n_tuples, statistics.mean(e2e_ms))
        e2e = {"value": e2e_tuples / (e2e_max / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_max, 2)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, wl["kind"], args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(max_ms / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32" if kb == 4 else "u64",
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": wl["desc"],
                           "closure_tuples": int(st.n_tuples), "iterations": int(iters),
                           "candidates": int(st.candidates), "edges": n,
                           "vertices": info["n_vertices"], "field_bits": info["field_bits"],
                           "l2": "flushed between steps (256 MB write); working set "
                                 + ("> L2" if 2 * kb * int(st.n_tuples) > (129 << 20) else "fits in L2"),
                           "parallelism": f"replicas x{world}", "regrows_timed": regrows,
                           "tiles": tiles or "compiled defaults"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(launches)}
        print(json.dumps(line))
    rel.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def autotune_ctx(ctx, rels, kind=None):
    """wg_autotune on the largest relation of each key width (outside every
    timed region); engines the context creates afterwards use the shapes."""
    from paper_2607_17571_gb300 import wg
    best = {}
    for i, r in enumerate(rels):
        info = r.info()
        kb = 4 if 2 * info["field_bits"] <= 32 else 8
        if kb not in best or info["n_edges"] > best[kb][1]:
            best[kb] = (i, info["n_edges"])
    out = {}
    for kb, (i, _) in sorted(best.items()):
        t = ctx.autotune(rels[i], wg.WG_TC if kind is None else kind)
        out[f"{kb}B_keys"] = {k: t[k] for k in ("count_tile", "emit_tile", "fuse_tile", "sort_mode",
                                                 "count_ms", "emit_ms", "fuse_ms", "sort_ms")}
    return out


def load_mix_golden(name, count):
    """{query index: oracle figures} from tests/golden/<name> (empty if absent)."""
    p = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(p):
        return {}
    qs = json.load(open(p))["queries"]
    return {i: q for i, q in enumerate(qs[:count])}


def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    return xs[min(len(xs) - 1, int(round(p / 100.0 * (len(xs) - 1))))]


def run_batch(args):
    """Many small uneven TC fixpoints: 4,096 ER queries (n log-uniform in
    [64, 16384], mean out-degree U[1.2, 3.0]), batched through wg_submit /
    wg_serve_step, against the plain per-query launch loop on the same GPU.
    One step = the whole set of queries in each arm."""
    import torch

    from paper_2607_17571_gb300 import inputs as I
    from paper_2607_17571_gb300 import wg

    torch.cuda.set_device(0)
    sizes = I.batch_query_sizes(args.n_queries)
    graphs = [I.er_graph(n, m, s) for (n, m, s) in sizes]
    ctx, rels = None, None

    def open_ctx():  # one context per arm, so neither holds the other's pools
        nonlocal ctx, rels
        if ctx is not None:
            for r in rels:
                r.free()
            ctx.close()
            torch.cuda.empty_cache()  # the next context's budget sees the memory again
        ctx = wg.Context(0)
        rels = [ctx.load(g.src, g.dst) for g in graphs]
        if not args.no_autotune:
            tuned.update(autotune_ctx(ctx, rels))
    tuned = {}
    # every query is checked against the oracle's closure size, iteration
    # count and digest of the sorted result (tests/golden/batch4096.json,
    # written by tests/golden/make_mix_golden.py, which calls only oracle/);
    # the device digests the result (wg_result_digest) so nothing is copied
    want = load_mix_golden("batch4096.json", len(graphs))

    failed = []

    def check(i, h, st):
        if st.state != wg.WG_DONE:
            failed.append({"query": i, "edges": int(sizes[i][1]), "error": int(st.error)})
            return 1
        g = want.get(i)
        if g is None:
            return 0
        return int(st.n_tuples != g["n_tuples"] or st.iterations != g["iterations"]
                   or h.digest() != int(g["digest"]))

    def batched():
        t0 = time.perf_counter()
        hs = ctx.submit([(wg.WG_TC, r) for r in rels])
        idx = {h.id: i for i, h in enumerate(hs)}
        lat, tuples, launches, bad, chk = [0.0] * len(hs), 0, 0, 0, 0.0
        left = len(hs)
        while left:
            ctx.serve_step(args.batch_iters)
            for qid in ctx.take_completed():
                i = idx[qid]
                h = hs[i]
                st = h.poll()
                lat[i] = (time.perf_counter() - t0 - chk) * 1e3
                tuples += st.n_tuples
                # checked and freed at once (a batched result stays in the
                # engine's result pool until freed); the check is not timed
                c0 = time.perf_counter()
                bad += check(i, h, st)
                h.free()
                chk += time.perf_counter() - c0
                left -= 1
        return time.perf_counter() - t0 - chk, lat, tuples, bad

    def plain():
        t0 = time.perf_counter()
        lat, tuples, launches, bad, chk = [], 0, 0, 0, 0.0
        for i, r in enumerate(rels):
            q = ctx.tc(r)
            try:
                st = q.wait()
            except wg.WgError:
                st = q.poll()
            lat.append((time.perf_counter() - t0 - chk) * 1e3)
            tuples += st.n_tuples
            launches += st.gpu_launches
            c0 = time.perf_counter()  # the check is not part of the loop's time
            bad += check(i, q, st)
            chk += time.perf_counter() - c0
            q.free()
        return time.perf_counter() - t0 - chk, lat, tuples, bad, launches

    # each arm: its own context, warmed up (engines, graphs, pools), then timed
    open_ctx()
    hs = ctx.submit([(wg.WG_TC, r) for r in rels[:32]])
    for h in hs:
        h.wait()
        h.free()
    ctx.take_completed()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    tb, lb, nb, bad_b = batched()
    clk_b = clocks.stop()
    open_ctx()
    for r in rels[:4]:
        q = ctx.tc(r)
        q.wait()
        q.free()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    tp, lp, npl, bad_p, launches = plain()
    clk_p = clocks.stop()
    n = len(rels)
    line = {"metric": "batched TC fixpoints: queries/s", "value": n / tb, "unit": "queries/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": round(tb * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "batch4096", "queries": n,
                       "desc": "ER TC queries, n log-uniform [64,16384], mean degree U[1.2,3.0], "
                               "seeds 40000+q", "closure_tuples_total": int(nb),
                       "iterations_per_launch": args.batch_iters,
                       "tiles": tuned or "compiled defaults"},
            "batched": {"seconds": round(tb, 3), "queries_per_s": n / tb, "tuples_per_s": nb / tb,
                        "p50_ms": _pct(lb, 50), "p99_ms": _pct(lb, 99), "parity_failures": bad_b,
                        "clocks": clk_b},
            "plain_loop": {"seconds": round(tp, 3), "queries_per_s": n / tp,
                           "tuples_per_s": npl / tp, "p50_ms": _pct(lp, 50), "p99_ms": _pct(lp, 99),
                           "parity_failures": bad_p, "gpu_launches": launches, "clocks": clk_p},
            "parity_checked": f"{len(want)} of {n} queries: closure size, iterations and "
                              "result digest against the oracle",
            "same_total": nb == npl, "failed_queries": failed[:20], "clocks": clk_b}
    print(json.dumps(line))
    for r in rels:
        r.free()
    ctx.close()
    return 0


def run_triangles(args):
    """Triangle counting (Sec. Generalization, "Triangle Counting") on an
    undirected R-MAT graph (2^16 nodes, 400k pairs = 800k directed edges)
    standing in for the paper's SNAP graphs.  One step = one wg_triangles call
    on the resident relation.  Its edges and CSR (~3.5 MB) live in L2, so the
    probe is latency-bound, not HBM-bound: the line reports milliseconds per
    count and two-paths probed per second, with no HBM roofline."""
    import torch

    import oracle
    from paper_2607_17571_gb300 import inputs as I
    from paper_2607_17571_gb300 import wg

    g = I.workload("tri_rmat16_800k")
    n = len(g)
    deg = np.bincount(g.src, minlength=int(max(g.src.max(), g.dst.max())) + 1)
    paths = int(deg[g.dst].astype(np.int64).sum())   # two-paths (a,b,c): sum of deg(b)
    if args.impl == "reference":  # the oracle as it stands, on the host cores
        threads = os.cpu_count()
        for _ in range(args.warmup if args.warmup < 1 else 1):
            oracle.oracle_triangles(g.src, g.dst, n_threads=threads)
        dts = []
        for _ in range(args.steps):
            t = time.perf_counter()
            want = oracle.oracle_triangles(g.src, g.dst, n_threads=threads)
            dts.append(time.perf_counter() - t)
        v = paths / statistics.mean(dts)
        print(json.dumps({"impl": "reference", "metric": "triangle count: two-paths probed/s",
                          "value": v, "unit": "two-paths/s", "n_gpus": 1, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(dts), 1),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "u64", "data": "synthetic",
                          "config": {"workload": "tri_rmat16_800k", "triangles": want},
                          "cpu_baseline": {"value": v, "unit": "two-paths/s", "cores": threads,
                                           "kind": "oracle", "sample": "whole count"},
                          "e2e": {"value": v, "unit": "two-paths/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    torch.cuda.set_device(0)
    ctx = wg.Context(0)
    stream = ctx.torch_stream
    rel = ctx.load(g.src, g.dst)
    count = None
    for _ in range(args.warmup):
        count = ctx.triangles(rel)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:0")
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ms = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        count = ctx.triangles(rel)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = statistics.mean(ms)
    # end to end: pinned edge list -> relation load -> count -> 8-byte result
    src_h, dst_h = wg.pinned(n, np.uint32), wg.pinned(n, np.uint32)
    src_h[:], dst_h[:] = g.src, g.dst
    e2e_ms = []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r2 = ctx.load(src_h, dst_h)
        c2 = ctx.triangles(r2)
        e2e_ms.append((time.perf_counter() - t) * 1e3)
        r2.free()
        assert c2 == count
    cpu = None
    if not args.no_cpu_baseline:
        threads = os.cpu_count()
        t = time.perf_counter()
        want = oracle.oracle_triangles(g.src, g.dst, n_threads=threads)
        dt = time.perf_counter() - t
        cpu = dict(value=paths / dt, unit="two-paths/s", cores=threads, kind="oracle",
                   sample=f"whole count ({want} triangles, {dt:.1f} s)", matches=want == count)
    e2e_mean = statistics.mean(e2e_ms)
    line = {"metric": "triangle count: two-paths probed/s", "value": paths / (t_ms / 1e3),
            "unit": "two-paths/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "tri_rmat16_800k",
                       "desc": "undirected R-MAT(.57,.19,.19,.05) 2^16 nodes, 400k distinct pairs "
                               "in both directions, seed 6", "edges": n,
                       "max_degree": int(deg.max()), "two_paths": paths, "triangles": count,
                       "l2": "flushed between steps (256 MB write); edges and CSR fit in L2"},
            "roofline": None,
            "e2e": {"value": paths / (e2e_mean / 1e3), "unit": "two-paths/s",
                    "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8,
                    "ms_per_step": round(e2e_mean, 2)},
            "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": 3 * args.steps}  # join count, partition, probe
    print(json.dumps(line))
    rel.free()
    ctx.close()
    return 0


def run_ablations(args):
    """The paper's engineering ablations (Sec. Evaluation: fused deduplication,
    the asynchronous loop, adaptive radix width, ping-pong buffers) on one TC
    workload: each variant is the same fixpoint with one design
    choice reverted, timed like the main bench (CUDA events, L2 flushed), and
    every variant's result is checked against the default's.  Variants:
    default (device loop, fused dedup/diff/merge, adaptive width, ping-pong),
    separate stages, host-driven loop (one launch per kernel, one host sync per
    iteration), host-driven loop with a readback and sync after every stage
    (the paper's stage-wise synchronisation), full-width radix sort, copy-back
    instead of ping-pong, and a
    linear-probing hash join in place of the sorted-array join (Sec. "Data
    Skew in Hash-Based Join"; its table is built once per relation, outside
    the timed steps)."""
    import torch

    from paper_2607_17571_gb300 import inputs as I
    from paper_2607_17571_gb300 import wg

    torch.cuda.set_device(0)
    name = args.ablate_workload
    g = I.workload(name)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:0")
    variants = [("default", {}), ("separate_stages", dict(separate_stages=True)),
                ("host_loop", dict(loop=wg.WG_LOOP_HOST)),
                ("host_staged", dict(loop=wg.WG_LOOP_HOST_STAGED)),
                ("full_width", dict(full_width=True)),
                ("merge_every_iter", dict(side_run="never")),
                ("copy_back", dict(copy_back=True)), ("hash_join", dict(hash_join=True))]
    ref, out = None, []
    clocks = Clocks(0)
    clocks.start()
    for vname, opts in variants:
        # one context per variant: its engine's pools are freed before the next
        ctx = wg.Context(0)
        stream = ctx.torch_stream
        rel = ctx.load(g.src, g.dst)
        q = ctx.tc(rel, **opts)
        q.wait()
        res = q.result()
        q.free()
        if ref is None:
            ref = res
        same = bool(np.array_equal(res, ref))
        for _ in range(max(0, args.warmup - 1)):
            q = ctx.tc(rel, **opts)
            q.wait()
            q.free()
        ms = []
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            q = ctx.tc(rel, **opts)
            st = q.wait()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            q.free()
        # the join's share (count + emit) from one profiled run: the paper's
        # "count-and-join time" of its hash vs binary-search comparison
        q = ctx.tc(rel, profile=True, **opts)
        q.wait()
        prof = {p["name"]: p["total_ms"] for p in q.profile()}
        q.free()
        out.append({"variant": vname, "ms": round(statistics.mean(ms), 3),
                    "tuples_per_s": st.n_tuples / (statistics.mean(ms) / 1e3),
                    "join_count_emit_ms": round(prof.get("join_count", 0.0) +
                                                prof.get("join_emit", 0.0), 3),
                    "same_result": same, "gpu_launches": st.gpu_launches})
        del res
        rel.free()
        ctx.close()
        torch.cuda.empty_cache()
    clk = clocks.stop()
    base = out[0]["ms"]
    for o in out:
        o["slowdown_vs_default"] = round(o["ms"] / base, 3)
    line = {"metric": "ablations: fixpoint ms per variant", "value": base, "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": base,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": name, "desc": WORKLOADS[name]["desc"],
                       "l2": "flushed between steps (256 MB write)"},
            "variants": out, "clocks": clk}
    print(json.dumps(line))
    return 0


def run_serve(args):
    """Open-loop Poisson arrivals of a mixed TC / SG request stream (see
    inputs.serve_request), served under a fixed device-memory budget: the
    continuous-batching server (requests join the running set at iteration
    boundaries) against the plain loop that runs one query at a time in
    arrival order.  Each rate offers --n-arrivals arrivals; arrival a asks
    for request a % pool of a pool of --n-requests distinct seeded requests
    (relations resident); each arm stops after --arm-seconds.  Every completed
    request is checked against the oracle's figures (closure size,
    iterations, result digest), outside the timed region."""
    import torch

    from paper_2607_17571_gb300 import inputs as I
    from paper_2607_17571_gb300 import wg

    torch.cuda.set_device(0)
    rates = [float(x) for x in args.rates.split(",")]
    reqs = [I.serve_request(r) for r in range(args.n_requests)]  # the pool
    kinds = [wg.WG_TC if k == "tc" else wg.WG_SG for k, _ in reqs]
    small = sorted(range(len(reqs)), key=lambda i: len(reqs[i][1]))[:6]
    # every completed request is checked against the oracle's closure size,
    # iteration count and result digest (tests/golden/serve_pool.json, written
    # by tests/golden/make_mix_golden.py, which calls only oracle/)
    want = load_mix_golden("serve_pool.json", len(reqs))
    npool = len(reqs)
    ctx, rels = None, None

    failed = []

    def check(i, h, st):
        if st.state != wg.WG_DONE:
            failed.append({"query": i, "edges": int(sizes[i][1]), "error": int(st.error)})
            return 1
        g = want.get(i)
        if g is None:
            return 0
        return int(st.n_tuples != g["n_tuples"] or st.iterations != g["iterations"]
                   or h.digest() != int(g["digest"]))

    def single(i):
        return (ctx.tc if kinds[i] == wg.WG_TC else ctx.sg)(rels[i])

    def open_ctx(batched_arm):
        """A fresh context under the budget for one arm (relations resident,
        warmed up on the smallest requests)."""
        nonlocal ctx, rels
        if ctx is not None:
            for r in rels:
                r.free()
            ctx.close()
            torch.cuda.empty_cache()
        ctx = wg.Context(0, mem_budget=int(args.budget_gb * (1 << 30)))
        rels = [ctx.load(g.src, g.dst) for _, g in reqs]
        if batched_arm:
            for h in ctx.submit([(kinds[i], rels[i]) for i in small]):
                h.wait()
                h.free()
            ctx.take_completed()
        else:
            for i in small:
                q = single(i)
                q.wait()
                q.free()

    def served(arr):
        # arrival a asks for pool request a % npool
        n = len(arr)
        lat, ok, rej, tuples, bad, chk = [None] * n, 0, 0, 0, 0, 0.0
        idx, nxt, done = {}, 0, 0
        t0 = time.perf_counter()
        while done < n and time.perf_counter() - t0 - chk < args.arm_seconds:
            now = time.perf_counter() - t0 - chk
            new = []
            while nxt < n and arr[nxt] <= now:
                new.append(nxt)
                nxt += 1
            if new:
                for a, h in zip(new, ctx.submit([(kinds[a % npool], rels[a % npool]) for a in new])):
                    idx[h.id] = (a, h)
            running = ctx.serve_step(args.serve_iters)
            t = time.perf_counter() - t0 - chk
            for qid in ctx.take_completed():
                a, h = idx.pop(qid)
                st = h.poll()
                lat[a] = (t - arr[a]) * 1e3
                if st.state == wg.WG_DONE:
                    ok += 1
                    tuples += st.n_tuples
                    c0 = time.perf_counter()  # the check is not part of the served time
                    bad += check(a % npool, h, st)
                    chk += time.perf_counter() - c0
                else:
                    rej += 1
                h.free()
                done += 1
            if running == 0 and nxt < n:
                time.sleep(max(0.0, min(0.002, arr[nxt] - (time.perf_counter() - t0 - chk))))
        el = time.perf_counter() - t0 - chk
        good = [x for x in lat if x is not None]
        unfinished = n - done  # closing the context waits only for the launch in flight
        return dict(seconds=round(el, 3), queries_per_s=ok / el, tuples_per_s=tuples / el,
                    p50_ms=_pct(good, 50), p99_ms=_pct(good, 99), completed=ok, rejected=rej,
                    unfinished_in_time=unfinished, parity_failures=bad)

    def plain(arr):
        n = len(arr)
        lat, ok, rej, tuples, bad, chk = [], 0, 0, 0, 0, 0.0
        t0 = time.perf_counter()
        for a in range(n):
            if time.perf_counter() - t0 - chk > args.arm_seconds:
                break
            wait = arr[a] - (time.perf_counter() - t0 - chk)
            if wait > 0:
                time.sleep(wait)
            q, st = None, None
            try:  # a query whose pools do not fit fails at the call or at the wait
                q = single(a % npool)
                st = q.wait()
                ok += 1
                tuples += st.n_tuples
            except wg.WgError:
                rej += 1
                st = None
            lat.append((time.perf_counter() - t0 - chk - arr[a]) * 1e3)
            if q is not None:
                if st is not None:
                    c0 = time.perf_counter()
                    bad += check(a % npool, q, st)
                    chk += time.perf_counter() - c0
                q.free()
        el = time.perf_counter() - t0 - chk
        return dict(seconds=round(el, 3), queries_per_s=ok / el, tuples_per_s=tuples / el,
                    p50_ms=_pct(lat, 50), p99_ms=_pct(lat, 99), completed=ok, rejected=rej,
                    unfinished_in_time=n - ok - rej, parity_failures=bad)

    points = []
    for rate in rates:
        arr = I.poisson_arrivals(args.n_arrivals, rate, seed=5)
        open_ctx(True)
        clocks = Clocks(0)
        clocks.start()
        b = served(arr)
        b["clocks"] = clocks.stop()
        open_ctx(False)
        clocks = Clocks(0)
        clocks.start()
        p = plain(arr)
        p["clocks"] = clocks.stop()
        points.append({"rate_qps": rate, "served": b, "plain_loop": p})
    best = max(points, key=lambda x: x["served"]["queries_per_s"])
    line = {"metric": "served TC/SG queries/s (p50/p99 latency)",
            "value": best["served"]["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
            "steps": len(rates), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": "serve", "arrivals_per_rate": args.n_arrivals,
                       "request_pool": npool, "arm_seconds_cap": args.arm_seconds,
                       "parity": f"every completed request: closure size, iterations and result "
                                 f"digest against the oracle ({len(want)} of {npool} pool "
                                 f"requests have oracle figures)",
                       "mix": "TC 75% (70% ER batch-mix sizes, 30% R-MAT DAG 1e4..1e6 edges), "
                              "SG 25% (forests, batch-mix sizes)",
                       "budget_gb": args.budget_gb, "iterations_per_round": args.serve_iters},
            "points": points}
    print(json.dumps(line))
    for r in rels:
        r.free()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the compiled tile shapes instead of running wg_autotune first")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tc_rmat17_400k",
                    choices=sorted(WORKLOADS) + ["batch4096", "serve", "tri_rmat16_800k",
                                                 "ablations"])
    ap.add_argument("--ablate-workload", default="tc_rmat17_400k", choices=sorted(WORKLOADS))
    ap.add_argument("--n-queries", type=int, default=4096)
    ap.add_argument("--batch-iters", type=int, default=4)
    ap.add_argument("--rates", default="100,200,500,1000,2000,5000")
    ap.add_argument("--n-requests", type=int, default=500,
                    help="served mix: distinct requests in the pool")
    ap.add_argument("--n-arrivals", type=int, default=10000,
                    help="served mix: arrivals per rate (arrival a asks for pool request a %% pool)")
    ap.add_argument("--budget-gb", type=float, default=60.0)
    ap.add_argument("--serve-iters", type=int, default=4)
    ap.add_argument("--arm-seconds", type=float, default=60.0,
                    help="wall-time limit of one serving arm at one rate")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--loop", default="device", choices=["device", "host", "staged"],
                    help="host: one launch per kernel and a host sync per iteration (profiling)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.workload == "batch4096":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "tri_rmat16_800k":
        return run_triangles(args)
    if args.workload == "ablations":
        return run_ablations(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
