#!/usr/bin/env python3
"""Benchmark of the Euler-tour hot path on one GB300 (or N, one process each).

One step = the whole path over one batch of synthetic inputs:
  * LCA at scale: three trees of n = 2^24 nodes (grasp unlimited, 1024 and 1,
    labels permuted), each preprocessed (Euler tour, list ranking, preorder /
    depth / size, sparse table) and then asked 2^24 uniform queries;
  * bridges: a small-diameter graph (n = 2^22, m = 2^25 - 1) and a
    large-diameter graph (n = 2^22, m = 2^22 - 1 + 2^24, 2^16 planted cuts).
value = (LCA queries + bridge edges) per second over the device-timed steps,
inputs resident in HBM. Per-part rates are in "breakdown".

--impl reference times the CPU oracle (test infrastructure, single thread) on
a bounded sample of the same workload; it is the reference arm of this
benchmark. With torchrun (N > 1) every rank runs its own replica of the
workload (weak scaling, no data-path collective); rank 0 prints the line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "LCA queries/s + bridge edges/s"
UNIT = "(queries+edges)/s"
TREES = [(1 << 24, None), (1 << 24, 1024), (1 << 24, 1)]
Q = 1 << 24
GRAPHS = [("easy", 1 << 22, (1 << 25) - 1), ("hard", 1 << 22, (1 << 22) - 1 + (1 << 24))]
WORKLOAD = ("LCA: 3 trees n=2^24 (grasp inf, 1024, 1; permuted labels) x (preprocess + 2^24 uniform queries); "
            "bridges: easy n=2^22 m=2^25-1, hard n=2^22 m=2^22-1+2^24 (2^16 planted cuts)")
SMALL_TREES = [(1 << 16, None)]
SMALL_Q = 1 << 16
SMALL_GRAPHS = [("easy", 1 << 14, 1 << 17), ("hard", 1 << 14, (1 << 14) - 1 + (1 << 16))]

# algorithmic bytes of the whole LCA path per node (blocked table) and per query (the per-step byte model)
LCA_PREPROCESS_BYTES_PER_NODE = 140
LCA_QUERY_BYTES = 40
E2E_MIN_STEPS = 60  # steps of the end-to-end measurement (at least --steps)

# algorithmic bytes per unit for each phase (what the method must read and write
# once: int32 = 4 B); keys are (phase, part) where part is "tree" or "graph"
ALGO = {
    ("rank.walk0", "tree"): ("arc", 12),       # read succ 4, write (sublist, offsets) 8
    ("rank.walk0", "graph"): ("arc", 12),
    ("rmq.level_min", "tree"): ("node", 8),    # read level l-1, write level l
    ("rmq.level_min", "graph"): ("pos", 8),
    ("rmq.level_max", "graph"): ("pos", 8),
    ("lca.query", "tree"): ("query", 32),      # u, v 8; pre of both 8; the two range entries 8; order 4; out 4
    ("lca.succ", "tree"): ("node", 16),        # child offsets 8, grouped child 4, successor 4 (per node)
    ("lca.node_rec", "tree"): ("node", 24),    # pre 4, size 4, (pm, sm) 8, record 8 of it used
    ("rmq.blocks", "tree"): ("node", 12),      # read Q, write pm and sm
    ("sort.scatter", "tree"): ("node", 16),    # read key, value; write key, value
    ("sort.scatter", "graph"): ("arc", 16),
    ("lca.node_stats", "tree"): ("node", 32),  # 2 records 16, write pre/depth/size 12, order 4
    ("lca.parent_pre", "tree"): ("node", 16),  # parent 4, pre 4, pre[parent] 4, Q 4
    ("br.hook", "graph"): ("edge", 17),        # edge 8, flag 1, two root lookups 8
    ("br.lowhigh_prep", "graph"): ("edge", 24),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="small sizes (functional check only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", choices=["all", "core", "batched", "serve", "methods"], default="all",
                    help="core = the scale workload; batched = 4096 mixed instances, batched vs per-instance")
    ap.add_argument("--case", choices=["lca", "easy", "hard", "batch_trees", "batch_graphs"], default=None,
                    help="run one workload of size --n twice (warm-up + one more) and exit; for profilers")
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--grasp", type=int, default=0, help="tree grasp for --case lca (0 = unlimited)")
    ap.add_argument("--seed", type=int, default=1,
                    help="seed of the step's synthetic inputs (rank r uses seed + r); the paper's protocol "
                         "repeats a measurement over five seeds")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t: float, world: int, device=None) -> float:
    """The slowest rank's time: the whole job is as fast as its slowest replica."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def step_stats(ms) -> dict:
    """Mean, standard deviation, minimum, median and maximum of per-step times (the statistics the
    paper reports over its repeated runs)."""
    ms = list(ms)
    return {"mean": statistics.mean(ms), "std": statistics.pstdev(ms), "min": min(ms),
            "median": statistics.median(ms), "max": max(ms), "n": len(ms)}


def replica_seed(rank: int, base: int = 1) -> int:
    """Each rank runs its own replica of the workload (weak scaling), with its own inputs."""
    return base + rank


# ------------------------------------------------------------------ inputs

def make_inputs(small: bool, seed: int):
    import synth
    trees = SMALL_TREES if small else TREES
    q = SMALL_Q if small else Q
    graphs = SMALL_GRAPHS if small else GRAPHS
    tr = []
    for n, grasp in trees:
        parent = synth.tree_parent(n, grasp, seed=seed)
        u, v = synth.lca_queries(n, q, seed=seed)
        tr.append(dict(n=n, grasp=grasp, parent=parent, u=u, v=v))
    gr = []
    for kind, n, m in graphs:
        if kind == "easy":
            e = synth.easy_graph(n, m, seed=seed)
        else:
            e = synth.hard_graph(n, m - (n - 1), max(1, n // 64), seed=seed)
        gr.append(dict(kind=kind, n=n, m=m, edges=e))
    return tr, gr


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch

    import paper_2103_15217_gb300 as etl

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    etl.build()
    etl.load_library()
    trees, graphs = make_inputs(args.small, seed=replica_seed(rank, args.seed))

    d_trees = [dict(t, parent_d=torch.from_numpy(t["parent"]).to(dev), u_d=torch.from_numpy(t["u"]).to(dev),
                    v_d=torch.from_numpy(t["v"]).to(dev)) for t in trees]
    d_graphs = [dict(g, edges_d=torch.from_numpy(g["edges"]).to(dev)) for g in graphs]
    units = sum(t["u"].shape[0] for t in trees) + sum(g["m"] for g in graphs)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step(record):
        """One pass of the whole path; record(name) drops an event on the stream."""
        outs = []
        for t in d_trees:
            record(f"tree{len(outs)}.start")
            h = etl.lca_preprocess(t["parent_d"])
            record(f"tree{len(outs)}.pre")
            out = h.query(t["u_d"], t["v_d"])
            record(f"tree{len(outs)}.query")
            h.free()
            outs.append(out)
        for g in d_graphs:
            record(f"graph.{g['kind']}.start")
            outs.append(etl.find_bridges(g["edges_d"], g["n"]))
            record(f"graph.{g['kind']}.end")
        return outs

    side = [torch.cuda.Stream() for _ in range(len(d_trees) + len(d_graphs))]

    def branches():
        """The instances of a step on parallel branches: each graph opens a branch and a tree follows
        it there (the last trees first), the remaining trees get a branch each. Three trees at once
        compete for L2 and DRAM; starting with the graphs, whose hooks and min / max passes work in
        L2, staggers them (measured 3% faster than one branch per instance, ~10% faster than one
        stream)."""
        tr = list(range(len(d_trees)))
        out = []
        for g in range(len(d_graphs)):
            out.append([("graph", g)] + ([("tree", tr.pop())] if tr else []))
        out += [[("tree", t)] for t in tr]
        return out

    layout = branches()

    def step_concurrent():
        """The same work as step(), on the parallel branches of branches(), each forked from and joined
        back into the current stream (one CUDA graph with parallel branches)."""
        main = torch.cuda.current_stream()
        outs = []
        for s_, branch in zip(side, layout):
            s_.wait_stream(main)
            with torch.cuda.stream(s_):
                for kind, i in branch:
                    if kind == "tree":
                        h = etl.lca_preprocess(d_trees[i]["parent_d"])
                        outs.append(h.query(d_trees[i]["u_d"], d_trees[i]["v_d"]))
                        h.free()
                    else:
                        outs.append(etl.find_bridges(d_graphs[i]["edges_d"], d_graphs[i]["n"]))
        for s_ in side[:len(layout)]:
            main.wait_stream(s_)
        return outs

    def timed_step(profile=False):
        evs = {}

        def rec(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            evs[name] = e
        step(rec)
        return evs

    for _ in range(args.warmup):
        flush.zero_()
        timed_step()
    torch.cuda.synchronize()

    # ---- eager steps with per-part events and the library's phase timers (breakdown + roofline)
    etl.profile_reset()
    etl.profile_enable(True)
    launches0 = etl.launch_count()
    steps = []
    for _ in range(args.steps):
        flush.zero_()
        steps.append(timed_step())
    torch.cuda.synchronize()
    launches_per_step = (etl.launch_count() - launches0) / args.steps
    etl.profile_enable(False)
    phases = etl.profile_read()

    # ---- the timed steps: the whole step captured once as a CUDA graph and replayed. The graph
    # runs the independent instances of a step on the parallel branches of branches() (forked
    # streams); the same step captured on one stream is timed too (sequential_graph_ms_per_step).
    def capture(fn):
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.graph(g, stream=cs):
            fn()
        torch.cuda.synchronize()
        return g

    seq_graph = capture(lambda: step(lambda name: None))
    seq_ts = []
    for _ in range(args.warmup + 3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seq_graph.replay()
        b.record(stream)
        b.synchronize()
        seq_ts.append(a.elapsed_time(b))
    t_seq_graph = statistics.median(seq_ts[args.warmup:]) / 1e3
    del seq_graph
    graph = capture(step_concurrent)
    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    replay_s = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        replay_s.append((a, b))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    replay_ms = [x.elapsed_time(y) for x, y in replay_s]
    t_graph = max_over_ranks(statistics.mean(replay_ms) / 1e3, world, dev)
    launches = int(round(launches_per_step * args.steps))
    del graph

    def el(evs, a, b):
        return evs[a].elapsed_time(evs[b]) / 1e3

    part = {}
    step_s = []
    for evs in steps:
        tot = 0.0
        for i, t in enumerate(trees):
            pre = el(evs, f"tree{i}.start", f"tree{i}.pre")
            qry = el(evs, f"tree{i}.pre", f"tree{i}.query")
            part.setdefault(f"tree{i}.pre", []).append(pre)
            part.setdefault(f"tree{i}.query", []).append(qry)
            tot += pre + qry
        for g in graphs:
            b = el(evs, f"graph.{g['kind']}.start", f"graph.{g['kind']}.end")
            part.setdefault(f"graph.{g['kind']}", []).append(b)
            tot += b
        step_s.append(tot)
    t_eager = max_over_ranks(sum(step_s) / len(step_s), world, dev)
    t_step = t_graph
    value = units * world / t_step

    breakdown = {}
    for i, t in enumerate(trees):
        pre = statistics.mean(part[f"tree{i}.pre"])
        qry = statistics.mean(part[f"tree{i}.query"])
        g = "inf" if t["grasp"] is None else str(t["grasp"])
        breakdown[f"lca_grasp_{g}"] = {
            "n": t["n"], "q": int(t["u"].shape[0]), "preprocess_ms": pre * 1e3, "query_ms": qry * 1e3,
            "preprocess_nodes_per_s": t["n"] / pre, "queries_per_s": t["u"].shape[0] / qry,
            "queries_per_s_incl_preprocess": t["u"].shape[0] / (pre + qry)}
    for g in graphs:
        b = statistics.mean(part[f"graph.{g['kind']}"])
        breakdown[f"bridges_{g['kind']}"] = {"n": g["n"], "m": g["m"], "ms": b * 1e3, "edges_per_s": g["m"] / b}

    roofline = roofline_from_phases(phases, trees, graphs, args.steps)
    if not args.small:
        roofline["random_access_ceiling"] = random_access_ceiling(etl, dev, flush)
        breakdown["lca_n16"] = small_tree_row(etl, dev, flush, args, seed=replica_seed(rank, args.seed))

    # ---- end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, etl, trees, graphs, dev, units, world)

    methods_res = run_methods(args, dev, trees) if args.mode == "all" else None
    if args.mode == "methods":
        methods_res = {"depth_sweep_n_2^23": run_methods(args, dev)}
    batched_res = run_batched(args, dev) if args.mode in ("all", "batched") else None
    serve_res = run_serve(args) if args.mode in ("all", "serve") else None
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded generators of the paper's tree and graph "
        "families; the bridge datasets of Table 1 are stood in for by the easy/hard generators)",
        "config": {"workload": WORKLOAD if not args.small else "small functional check", "units_per_step": units,
                   "timing": "each step is one CUDA-graph replay of the whole path (captured once); "
                             "breakdown and phase timers come from the same number of eager (sequential) steps",
                   "seed": replica_seed(rank, args.seed),
                   "step_ms_stats": step_stats(replay_ms),
                   "eager_ms_per_step": t_eager * 1e3,
                   "sequential_graph_ms_per_step": t_seq_graph * 1e3,
                   "concurrency": "the step runs on parallel graph branches: " + " | ".join(
                       " then ".join(f"{k} {i}" for k, i in b) for b in layout),
                   "l2": "flushed between steps (512 MB write) and working set >> L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "wall_s_timed": wall},
        "breakdown": breakdown,
        "lca_methods": methods_res,
        "batched": batched_res,
        "serving": serve_res,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in sorted(phases.items())},
        "phase_rooflines": phase_rooflines(phases, trees, graphs, args.steps),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(trees, graphs)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result if rank == 0 else None


def random_access_ceiling(etl, dev, flush, n=1 << 25, reps=5):
    """A measured ceiling for the ranking walk. The probe kernel performs the walk's accesses (a
    random 4-byte successor read and an 8-byte record write at the same index) for every element of
    a random permutation of 2^25 elements, all independent of one another; the library's ranker then
    ranks the list that visits the elements in that same order, where each step's read depends on the
    previous one. Both run with 512 MB flushed from L2 before each launch; the fraction is the probe's
    time over the level-0 walk's (k_walk0) time on the same list: the same elements, the same random
    addresses."""
    import torch
    order = torch.randperm(n, device=dev, dtype=torch.int32)
    succ = torch.empty(n, dtype=torch.int32, device=dev)
    succ[order[:-1].long()] = order[1:]
    succ[order[-1].long()] = -1
    out = torch.empty(n, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    ts = []
    for i in range(reps + 2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        etl.probe_gather_scatter(order, succ, out)
        b.record(stream)
        b.synchronize()
        if i >= 2:
            ts.append(a.elapsed_time(b) / 1e3)
    t_probe = statistics.median(ts)
    head = int(order[0].item())
    etl.list_rank(succ, head)  # warm-up
    torch.cuda.synchronize()
    walk = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        etl.profile_reset()
        etl.profile_enable(True)
        etl.list_rank(succ, head)
        etl.profile_enable(False)
        walk.append(etl.profile_read()["rank.walk0"][0] / 1e3)
    t_walk = statistics.median(walk)
    etl.profile_reset()
    del order, succ, out
    return {"probe_kernel": "k_probe_gather_scatter", "elements": n,
            "probe_ms": t_probe * 1e3, "probe_elements_per_s": n / t_probe,
            "probe_algorithmic_gbs": 12 * n / t_probe / 1e9,
            "walk_ms": t_walk * 1e3, "walk_elements_per_s": n / t_walk,
            "walk_frac_of_ceiling": t_probe / t_walk,
            "note": "same random list for both: the probe does every element's 4 B gather + 8 B scatter "
                    "independently, the walk follows the list (dependent loads); L2 flushed before each"}


def small_tree_row(etl, dev, flush, args, seed, n=1 << 16, q=1 << 16):
    """The small LCA configuration: one random recursive tree of 2^16 nodes (labels permuted) and 2^16
    uniform queries, preprocessing and queries timed separately, eagerly and as captured CUDA graphs
    (at this size launch overhead, not HBM, bounds the time)."""
    import torch

    import synth
    parent = torch.from_numpy(synth.tree_parent(n, None, seed=seed)).to(dev)
    u, v = (torch.from_numpy(x).to(dev) for x in synth.lca_queries(n, q, seed=seed))
    out = torch.empty_like(u)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    reps = max(5, args.steps)
    res = {"n": n, "q": q}
    with torch.cuda.stream(stream):
        h = etl.lca_preprocess(parent)
        h.query(u, v, out=out)
        torch.cuda.synchronize()
        pre_ms, qry_ms = [], []
        l0 = etl.launch_count()
        for _ in range(reps):
            flush.zero_()
            h.free()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            h = etl.lca_preprocess(parent)
            b.record(stream)
            h.query(u, v, out=out)
            c.record(stream)
            c.synchronize()
            pre_ms.append(a.elapsed_time(b))
            qry_ms.append(b.elapsed_time(c))
        res["launches_per_preprocess_and_query"] = (etl.launch_count() - l0) / reps
        h.free()
        # the captured preprocessing keeps its tables in a caller-owned workspace, so the graph holds no
        # allocation that would outlive a replay
        ws = etl.new_workspace(etl.workspace_size("lca_preprocess", n), device=dev)
        gp, gq = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gp, stream=stream):
            hg = etl.lca_preprocess(parent, workspace=ws)
        with torch.cuda.graph(gq, stream=stream):
            hg.query(u, v, out=out)
        gpre, gqry = [], []
        for _ in range(reps + 2):
            flush.zero_()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            gp.replay()
            b.record(stream)
            gq.replay()
            c.record(stream)
            c.synchronize()
            gpre.append(a.elapsed_time(b))
            gqry.append(b.elapsed_time(c))
        gpre, gqry = gpre[2:], gqry[2:]
        hg.free()
        del gp, gq
    peak, _ = _peak_hbm()
    pre_s, qry_s = statistics.median(pre_ms) / 1e3, statistics.median(qry_ms) / 1e3
    gpre_s, gqry_s = statistics.median(gpre) / 1e3, statistics.median(gqry) / 1e3
    res.update({
        "preprocess_ms": pre_s * 1e3, "query_ms": qry_s * 1e3,
        "preprocess_nodes_per_s": n / pre_s, "queries_per_s": q / qry_s,
        "graph_preprocess_ms": gpre_s * 1e3, "graph_query_ms": gqry_s * 1e3,
        "graph_preprocess_nodes_per_s": n / gpre_s, "graph_queries_per_s": q / gqry_s,
        "hbm_frac_preprocess": LCA_PREPROCESS_BYTES_PER_NODE * n / gpre_s / 1e9 / peak,
        "hbm_frac_query": LCA_QUERY_BYTES * q / gqry_s / 1e9 / peak,
        "bytes_model": f"{LCA_PREPROCESS_BYTES_PER_NODE} B/node preprocessing, {LCA_QUERY_BYTES} B/query "
                       "(algorithmic, blocked table)",
        "timing": "median of repeated runs, L2 flushed before each; eager (public API calls) and captured "
                  "graph replays"})
    return res


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("hbm_gbs")
    except Exception:
        peak = None
    return (peak, "measured") if peak else (6800.0, "fallback")


def algorithmic_bytes_per_launch(name, trees, graphs):
    """Algorithmic bytes one launch of phase `name` moves on this workload (the per-unit figure of
    ALGO times the units of one instance), or None if the phase has no per-unit figure. A phase
    that both parts run is averaged over one launch per instance."""
    n_tree, n_graph = len(trees), len(graphs)
    tree_units = {"node": sum(t["n"] for t in trees) / max(n_tree, 1),
                  "arc": sum(2 * t["n"] for t in trees) / max(n_tree, 1),
                  "query": sum(t["u"].shape[0] for t in trees) / max(n_tree, 1)}
    graph_units = {"edge": sum(g["m"] for g in graphs) / max(n_graph, 1),
                   "arc": sum(2 * g["n"] - 1 for g in graphs) / max(n_graph, 1),
                   "pos": sum(2 * g["n"] - 1 for g in graphs) / max(n_graph, 1)}
    kt, kg = ALGO.get((name, "tree")), ALGO.get((name, "graph"))
    if kt and kg:
        return (n_tree * tree_units[kt[0]] * kt[1] + n_graph * graph_units[kg[0]] * kg[1]) / (n_tree + n_graph)
    if kt:
        return tree_units[kt[0]] * kt[1]
    if kg:
        return graph_units[kg[0]] * kg[1]
    return None


def phase_rooflines(phases, trees, graphs, steps):
    """Every timed phase with a per-unit byte figure: its algorithmic bytes per launch, average
    launch time and the bandwidth that makes, against the measured copy peak."""
    peak, _ = _peak_hbm()
    out = {}
    for name, (ms, launches) in sorted(phases.items()):
        b = algorithmic_bytes_per_launch(name, trees, graphs)
        if b is None or not launches or ms <= 0:
            continue
        avg_s = ms / 1e3 / launches
        out[name] = {"ms_per_step": ms / steps, "launches_per_step": launches / steps, "bytes_per_launch": b,
                     "avg_launch_ms": avg_s * 1e3, "achieved_gbs": b / avg_s / 1e9, "frac": b / avg_s / 1e9 / peak}
    return out


def roofline_from_phases(phases, trees, graphs, steps):
    peak, peak_src = _peak_hbm()
    # dominant phase by total device time
    name, (ms, launches) = max(phases.items(), key=lambda kv: kv[1][0])
    bytes_per_launch = algorithmic_bytes_per_launch(name, trees, graphs)
    if bytes_per_launch is None:
        return {"bound": "hbm", "kernel": name, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "note": "no algorithmic byte count for this phase"}
    avg_s = ms / 1e3 / launches
    achieved = bytes_per_launch / avg_s / 1e9
    traffic = committed_traffic(name, len(trees), len(graphs))
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
            "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_s * 1e3, "launches_per_step": launches / steps}


def committed_traffic(phase: str, n_trees: int, n_graphs: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu capture
    (profiles/k_walk0_traffic.json), or None if that capture is for another kernel,
    another workload, an older version of the kernel's source or other launch parameters."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "k_walk0_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except Exception:
        return None
    if rec.get("phase") != phase or rec.get("source_sha256") != sha or (n_trees, n_graphs) != (3, 2):
        return None
    import paper_2103_15217_gb300 as etl
    tuned = etl.tune_get()
    if any(tuned.get(k) != v for k, v in rec.get("launch_params", {}).items()):
        return None  # the capture was taken with other launch parameters
    c = rec["cases"]
    keys = ("lca_grasp_inf", "lca_grasp_1024", "lca_grasp_1", "easy", "hard")  # one walk launch each per step
    if any(k not in c for k in keys):
        return None
    return sum(c[k]["traffic_bytes"] for k in keys) / len(keys)


def run_e2e(args, etl, trees, graphs, dev, units, world):
    import torch
    stream = torch.cuda.current_stream()
    h_trees = [dict(parent=torch.from_numpy(t["parent"]).pin_memory(), u=torch.from_numpy(t["u"]).pin_memory(),
                    v=torch.from_numpy(t["v"]).pin_memory(),
                    out=torch.empty(t["u"].shape[0], dtype=torch.int32).pin_memory(), n=t["n"]) for t in trees]
    h_graphs = [dict(edges=torch.from_numpy(g["edges"]).pin_memory(),
                     out=torch.empty(g["m"], dtype=torch.uint8).pin_memory(), n=g["n"]) for g in graphs]
    h2d = sum(t["parent"].numel() * 4 + t["u"].numel() * 8 for t in h_trees) + sum(g["edges"].numel() * 4 for g in h_graphs)
    d2h = sum(t["out"].numel() * 4 for t in h_trees) + sum(g["out"].numel() for g in h_graphs)

    # device buffers for the inputs and results, allocated once: every step copies its inputs into
    # them and its results out of them (a fresh allocation per step would make the caching allocator
    # call cudaMalloc whenever a block is still held by another stream, a stall of tens of ms)
    # and each instance's scratch (and a tree's tables) in a workspace of its own, sized by the library
    # and laid out once: no step asks an allocator for memory, so no step waits for one to map more
    for x in h_trees:
        x["d"] = {k: torch.empty_like(x[k], device=dev) for k in ("parent", "u", "v", "out")}
        x["ws"] = etl.new_workspace(etl.workspace_size("lca_preprocess", x["n"]), device=dev)
    for x in h_graphs:
        x["d"] = {k: torch.empty_like(x[k], device=dev) for k in ("edges", "out")}
        x["ws"] = etl.new_workspace(etl.workspace_size("find_bridges", x["n"], x["edges"].shape[0]), device=dev)

    def tree_job(t):
        d = t["d"]
        d["parent"].copy_(t["parent"], non_blocking=True)
        d["u"].copy_(t["u"], non_blocking=True)
        d["v"].copy_(t["v"], non_blocking=True)
        h = etl.lca_preprocess(d["parent"], workspace=t["ws"])
        h.query(d["u"], d["v"], out=d["out"])
        t["out"].copy_(d["out"], non_blocking=True)
        h.free()

    def graph_job(g):
        d = g["d"]
        d["edges"].copy_(g["edges"], non_blocking=True)
        etl.find_bridges(d["edges"], g["n"], out=d["out"], workspace=g["ws"])
        g["out"].copy_(d["out"], non_blocking=True)

    jobs = [(tree_job, t) for t in h_trees] + [(graph_job, g) for g in h_graphs]
    side = [torch.cuda.Stream() for _ in jobs]
    copy_side = [torch.cuda.Stream() for _ in h_trees]

    def one_sequential():
        for fn, x in jobs:
            fn(x)

    def one_pipelined():
        """Each instance on its own stream. The inputs that computation starts from (parent arrays,
        edge lists) are copied first; the query pairs follow on separate copy streams while the trees
        are being preprocessed, and each tree's queries wait only for their own pairs. Results are
        copied out on the instance's stream."""
        handles = []
        for s_, t in zip(side, h_trees):
            s_.wait_stream(stream)
            with torch.cuda.stream(s_):
                t["d"]["parent"].copy_(t["parent"], non_blocking=True)
                handles.append(etl.lca_preprocess(t["d"]["parent"], workspace=t["ws"]))
        for s_, g in zip(side[len(h_trees):], h_graphs):
            s_.wait_stream(stream)
            with torch.cuda.stream(s_):
                graph_job(g)
        for s_, cs, t, h in zip(side, copy_side, h_trees, handles):
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                t["d"]["u"].copy_(t["u"], non_blocking=True)
                t["d"]["v"].copy_(t["v"], non_blocking=True)
            s_.wait_stream(cs)
            with torch.cuda.stream(s_):
                h.query(t["d"]["u"], t["d"]["v"], out=t["d"]["out"])
                t["out"].copy_(t["d"]["out"], non_blocking=True)
                h.free()
        for s_ in side + copy_side:
            stream.wait_stream(s_)

    host_s = []

    def timed(one, steps):
        for _ in range(max(1, args.warmup)):
            one()
        torch.cuda.synchronize()
        host_s.clear()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for i in range(steps):
            h0 = time.perf_counter()
            one()
            host_s.append(time.perf_counter() - h0)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        return evs[0].elapsed_time(evs[-1]) / 1e3 / steps, per

    # at least E2E_MIN_STEPS steps: on some boxes one step in a few dozen takes tens of ms longer (the
    # device-resident graph replays never do), and the mean over more steps weighs such a pause as
    # often as it occurs instead of by the luck of a short run
    e2e_steps = max(args.steps, E2E_MIN_STEPS)
    t_seq, _ = timed(one_sequential, args.steps)
    t_seq = max_over_ranks(t_seq, world, dev)
    t, per_step = timed(one_pipelined, e2e_steps)
    t = max_over_ranks(t, world, dev)
    # copy bandwidth alone, for context: every input of a step in, every result out, nothing else
    dsts = [torch.empty_like(x[k], device=dev) for _, x in jobs for k in ("parent", "u", "v", "edges") if k in x]
    srcs = [x[k] for _, x in jobs for k in ("parent", "u", "v", "edges") if k in x]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(4):
        if i == 1:
            a.record(stream)
        for d_, s_ in zip(dsts, srcs):
            d_.copy_(s_, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    h2d_s = a.elapsed_time(b) / 1e3 / 3
    del dsts
    return {"value": units * world / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": t * 1e3, "steps": e2e_steps, "sequential_ms_per_step": t_seq * 1e3,
            "step_ms_min_median_max": [min(per_step), statistics.median(per_step), max(per_step)],
            "step_ms": per_step,
            "host_enqueue_ms_per_step": 1e3 * statistics.median(host_s),
            "host_enqueue_ms_max": 1e3 * max(host_s),
            "h2d_only_ms_per_step": h2d_s * 1e3, "h2d_gb_per_s": h2d / h2d_s / 1e9,
            "timing": "public API calls, eager; each instance on its own stream (copy in, compute, copy out), "
                      "query pairs copied on side streams during preprocessing; host inputs pinned; each "
                      "instance's scratch in a caller-owned workspace (the _ws entry points)"}


# ------------------------------------------------------------------ batched instances

def make_batch_inputs(small: bool, seed: int = 1):
    import synth
    from synth.generators import make_graph, make_tree
    nt, ng = (64, 64) if small else (2048, 2048)
    trees, graphs = synth.batched_instances(seed=seed, ntrees=nt, ngraphs=ng)
    tp, tu, tv, ti, toff = [], [], [], [], [0]
    for i, d in enumerate(trees):
        p, u, v = make_tree(d)
        tp.append(p)
        tu.append(u)
        tv.append(v)
        ti.append(np.full(u.shape[0], i, np.int32))
        toff.append(toff[-1] + d["n"])
    ge, eoff, noff = [], [0], [0]
    for d in graphs:
        e = make_graph(d)
        ge.append(e)
        eoff.append(eoff[-1] + e.shape[0])
        noff.append(noff[-1] + d["n"])
    return dict(trees=trees, graphs=graphs, tp=tp, tu=tu, tv=tv, ti=ti, toff=np.array(toff, np.int32),
                ge=ge, eoff=np.array(eoff, np.int32), noff=np.array(noff, np.int32))


def run_batched(args, dev):
    """Per-instance launches vs one batched, graph-captured launch sequence (equal results required)."""
    import torch

    import paper_2103_15217_gb300 as etl
    B = make_batch_inputs(args.small)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    tp = [T(x) for x in B["tp"]]
    tu = [T(x) for x in B["tu"]]
    tv = [T(x) for x in B["tv"]]
    ge = [T(x) for x in B["ge"]]
    P, O = T(np.concatenate(B["tp"])), T(B["toff"])
    I, U, V = T(np.concatenate(B["ti"])), T(np.concatenate(B["tu"])), T(np.concatenate(B["tv"]))
    E, EO, NO = T(np.concatenate(B["ge"])), T(B["eoff"]), T(B["noff"])
    max_n = max(d["n"] for d in B["trees"])
    total_gn = int(B["noff"][-1])
    q_total, m_total = int(U.numel()), int(E.shape[0])
    units = q_total + m_total
    outs_pi = [torch.empty_like(u) for u in tu]
    masks_pi = [torch.empty(e.shape[0], dtype=torch.uint8, device=dev) for e in ge]
    out_b = torch.empty_like(U)
    mask_b = torch.empty(m_total, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def per_instance():
        for i in range(len(tp)):
            h = etl.lca_preprocess(tp[i])
            h.query(tu[i], tv[i], out=outs_pi[i])
            h.free()
        for i, d in enumerate(B["graphs"]):
            masks_pi[i].copy_(etl.find_bridges(ge[i], d["n"]))

    from paper_2103_15217_gb300 import tune
    defaults = etl.tune_get()

    def batched_trees():
        h = etl.lca_preprocess_batch(P, O, max_n)
        h.query_batch(I, U, V, out=out_b)
        h.free()

    def batched_graphs():
        mask_b.copy_(etl.find_bridges_batch(E, EO, NO, total_gn))

    def batched():
        """The tree batch, then the graph batch, on one stream: side by side on two streams they
        measured 3.5% slower (both are bound by memory traffic and only contend for it)."""
        batched_trees()
        batched_graphs()

    def one(fn=None, graph=None):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay() if graph is not None else fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                g.replay()
        torch.cuda.synchronize()
        return g

    def timed_graphs(graphs, reps):
        """Replays of several captured graphs, interleaved so that drift of the box hits all alike;
        per graph the mean and the median (seconds)."""
        ts = [[] for _ in graphs]
        with torch.cuda.stream(stream):
            for _ in range(reps):
                for k, g in enumerate(graphs):
                    ts[k].append(one(graph=g))
        return [(statistics.mean(t), statistics.median(t)) for t in ts]

    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        per_instance()
        batched()
    torch.cuda.synchronize()
    equal = bool(torch.equal(torch.cat(outs_pi), out_b) and torch.equal(torch.cat(masks_pi), mask_b))

    # the batch captured with the default launch parameters, then the autotuner on this very mix
    # (eager runs of the batch), then the batch captured again with the tuned parameters; the two
    # graphs are timed alternately
    g_def = capture(batched)
    with torch.cuda.stream(stream):
        tuned = tune.autotune(batched, key=f"batched {len(tp)} trees + {len(ge)} graphs", use_cache=False)
    torch.cuda.synchronize()
    g = capture(batched)
    with torch.cuda.stream(stream):
        t_pi = statistics.median(one(fn=per_instance) for _ in range(max(1, min(args.steps, 3))))
    l0 = etl.launch_count()
    (def_mean, def_med), (t_mean, t_med) = timed_graphs([g_def, g], args.steps)
    launches_b = etl.launch_count() - l0  # graph replays do not go through the library's launch sites
    g.replay()
    torch.cuda.synchronize()
    equal = equal and bool(torch.equal(torch.cat(outs_pi), out_b) and torch.equal(torch.cat(masks_pi), mask_b))
    del g, g_def
    parts = {}
    for name, fn in (("trees", batched_trees), ("graphs", batched_graphs)):
        gp = capture(fn)
        parts[name + "_ms"] = timed_graphs([gp], args.steps)[0][1] * 1e3
        del gp
    etl.tune_set(**defaults)
    return {
        "autotuned": {"params": tuned["params"], "defaults": defaults, "trials": tuned["trials"],
                      "tuned_on": "eager runs of this batch (the whole mix of trees and graphs)",
                      "eager_default_ms": tuned["default_ms"], "eager_tuned_ms": tuned["ms"],
                      "graph_default_ms": def_med * 1e3, "graph_tuned_ms": t_med * 1e3,
                      "graph_gain": def_med / t_med,
                      "timing": "medians of alternating replays of the two captured graphs"},
        "workload": (f"{len(tp)} trees n log-uniform 2^6..2^18 (grasp 1, 1024, inf round robin) with n queries each"
                     f" + {len(ge)} graphs n log-uniform 2^6..2^16, m = 4n (easy/hard alternating)"),
        "queries": q_total, "edges": m_total, "tree_nodes": int(B["toff"][-1]), "graph_nodes": total_gn,
        "per_instance": {"ms": t_pi * 1e3, "value": units / t_pi},
        "batched_graph": {"ms": t_mean * 1e3, "median_ms": t_med * 1e3, "value": units / t_mean, "captured": True,
                          "concurrency": "tree batch then graph batch on one stream", "alone": parts},
        "speedup": t_pi / t_mean, "results_identical": equal, "unit": UNIT,
        "host_launch_sites_during_replay": launches_b,
    }


# ------------------------------------------------------------------ LCA methods

def _median_ms(fn, reps=3):
    import torch
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def compare_methods(parent_np, u_np, v_np, dev, naive_step_budget=2e9):
    """RMQ (this path), Inlabel (the paper's GPU method) and naive climbing (the paper's
    comparison method) on one tree: preprocessing and query times, answers cross-checked."""
    import torch

    import paper_2103_15217_gb300 as etl
    n, q = parent_np.shape[0], u_np.shape[0]
    P = torch.from_numpy(parent_np).to(dev)
    U, V = torch.from_numpy(u_np).to(dev), torch.from_numpy(v_np).to(dev)
    res = {"n": n, "q": q}
    h = etl.lca_preprocess(P)
    h.build_inlabel(P)
    torch.cuda.synchronize()

    def pre_rmq():
        x = etl.lca_preprocess(P)
        x.free()

    def pre_inl():
        x = etl.lca_preprocess(P, methods=("inlabel",))
        x.free()

    def pre_tour():
        x = etl.lca_preprocess(P, methods=("tour_rmq",))
        x.free()
    t_rmq_pre = _median_ms(pre_rmq)
    t_inl_pre = _median_ms(pre_inl)
    t_tour_pre = _median_ms(pre_tour)
    ht = etl.lca_preprocess(P, methods=("tour_rmq",))
    out_t = torch.empty_like(U)
    t_tour_q = _median_ms(lambda: ht.query_tour(U, V, out=out_t))
    ht.free()
    out_r = torch.empty_like(U)
    out_i = torch.empty_like(U)
    t_rmq_q = _median_ms(lambda: h.query(U, V, out=out_r))
    t_inl_q = _median_ms(lambda: h.query_inlabel(U, V, out=out_i))
    depth_mean = float(h.arrays()["depth"].double().mean().item())
    # naive: full query set unless its climbs would exceed the step budget; then a prefix sample
    qn = int(min(q, max(1024, naive_step_budget / max(1.0, 2 * depth_mean))))
    nv = etl.NaiveLca(P)
    t_nv_pre = _median_ms(lambda: etl.NaiveLca(P))
    out_n = torch.empty(qn, dtype=torch.int32, device=dev)
    t_nv_q = _median_ms(lambda: nv.query(U[:qn], V[:qn], out=out_n), reps=2)
    # the same RMQ method on a full sparse table (n log n entries) instead of the blocked one
    blocked0 = etl.tune_get()["rmq_blocked"]
    etl.tune_set(rmq_blocked=0)
    try:
        hf = etl.lca_preprocess(P)
        out_f = torch.empty_like(U)
        t_full_pre = _median_ms(pre_rmq)
        t_full_q = _median_ms(lambda: hf.query(U, V, out=out_f))
        hf.free()
    finally:
        etl.tune_set(rmq_blocked=blocked0)
    agree = bool(torch.equal(out_r, out_i) and torch.equal(out_r[:qn], out_n) and torch.equal(out_r, out_f)
                 and torch.equal(out_r, out_t))
    h.free()
    res.update({
        "avg_depth": depth_mean,
        "rmq": {"preprocess_ms": t_rmq_pre, "query_ms": t_rmq_q, "queries_per_s": q / t_rmq_q * 1e3,
                "table": "blocked" if blocked0 else "full"},
        "rmq_full_table": {"preprocess_ms": t_full_pre, "query_ms": t_full_q, "queries_per_s": q / t_full_q * 1e3},
        "rmq_euler_tour": {"preprocess_ms": t_tour_pre, "query_ms": t_tour_q, "queries_per_s": q / t_tour_q * 1e3},
        "inlabel": {"preprocess_ms": t_inl_pre, "query_ms": t_inl_q, "queries_per_s": q / t_inl_q * 1e3},
        "naive": {"preprocess_ms": t_nv_pre, "queries_timed": qn, "query_ms_for_timed": t_nv_q,
                  "queries_per_s": qn / t_nv_q * 1e3, "query_ms_for_all_q_est": t_nv_q * q / qn},
        "answers_identical": agree,
    })
    return res


def compare_bridge_methods(edges_np, n, dev):
    """Tarjan-Vishkin (this path) against the paper's hybrid (tour levels + CK marking)."""
    import torch

    import paper_2103_15217_gb300 as etl
    E = torch.from_numpy(edges_np).to(dev)
    a = etl.find_bridges(E, n)
    b = etl.find_bridges(E, n, method="hybrid")
    torch.cuda.synchronize()
    t_tv = _median_ms(lambda: etl.find_bridges(E, n))
    t_hy = _median_ms(lambda: etl.find_bridges(E, n, method="hybrid"))
    blocked0 = etl.tune_get()["rmq_blocked"]
    etl.tune_set(rmq_blocked=0)
    try:
        c = etl.find_bridges(E, n)
        t_full = _median_ms(lambda: etl.find_bridges(E, n))
    finally:
        etl.tune_set(rmq_blocked=blocked0)
    m = edges_np.shape[0]
    return {"n": n, "m": m, "tv_ms": t_tv, "hybrid_ms": t_hy, "tv_full_tables_ms": t_full,
            "tv_edges_per_s": m / t_tv * 1e3, "hybrid_edges_per_s": m / t_hy * 1e3,
            "masks_identical": bool(torch.equal(a, b) and torch.equal(a, c))}


def run_methods(args, dev, trees=None):
    """Three n = 2^24 trees of the main workload, or (mode methods) the depth sweep of Sec. 3.3."""
    import synth
    out = {}
    if trees is not None:
        for t in trees:
            g = "inf" if t["grasp"] is None else str(t["grasp"])
            out[f"grasp_{g}"] = compare_methods(t["parent"], t["u"], t["v"], dev)
        return out
    for kind, n in (("easy", 1 << 20), ("hard", 1 << 20), ("easy", 1 << 22), ("hard", 1 << 22)):
        if args.small:
            n = 1 << 14
        e = synth.easy_graph(n, 8 * n, seed=5) if kind == "easy" else synth.hard_graph(n, 4 * n, n // 64, seed=5)
        out[f"bridges_{kind}_n{n}"] = compare_bridge_methods(e, n, dev)
    # scale-free trees (Sec. 3.3, "Scale-Free Trees")
    nb = 1 << 21 if not args.small else 1 << 14
    parent = synth.ba_tree(nb, seed=3)
    u, v = synth.lca_queries(nb, nb, seed=3)
    out[f"barabasi_albert_n{nb}"] = compare_methods(parent, u, v, dev)
    n = 1 << 23 if not args.small else 1 << 16
    for grasp in (None, 100000, 10000, 1000, 100, 10, 1):
        parent = synth.tree_parent(n, grasp, seed=3)
        u, v = synth.lca_queries(n, n, seed=3)
        g = "inf" if grasp is None else str(grasp)
        out[f"grasp_{g}"] = compare_methods(parent, u, v, dev)
    out["queries_to_nodes"] = queries_to_nodes(n, dev)
    out["batch_size"] = batch_size_sweep(n, dev, small=args.small)
    return out


def queries_to_nodes(n, dev):
    """Total time (preprocessing + all queries) against the queries-to-nodes ratio on a shallow tree
    (the experiment of Sec. 3.3, "Queries to Nodes Ratio"): RMQ, Inlabel and the naive method."""
    import torch

    import paper_2103_15217_gb300 as etl
    import synth
    P = torch.from_numpy(synth.tree_parent(n, None, seed=4)).to(dev)
    qmax = 16 * n
    u, v = synth.lca_queries(n, qmax, seed=4)
    U, V = torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev)
    out_r = torch.empty_like(U)
    out_i = torch.empty_like(U)
    out_n = torch.empty_like(U)
    res = {"n": n, "tree": "random recursive (shallow)", "rows": []}
    agree = True
    for ratio in (0.125, 0.25, 0.5, 1, 2, 4, 8, 16):
        q = int(n * ratio)

        def rmq():
            h = etl.lca_preprocess(P)
            h.query(U[:q], V[:q], out=out_r[:q])
            h.free()

        def inl():
            h = etl.lca_preprocess(P, methods=("inlabel",))
            h.query_inlabel(U[:q], V[:q], out=out_i[:q])
            h.free()

        def naive():
            etl.NaiveLca(P).query(U[:q], V[:q], out=out_n[:q])
        rmq(), inl(), naive()
        torch.cuda.synchronize()
        agree = agree and bool(torch.equal(out_r[:q], out_i[:q]) and torch.equal(out_r[:q], out_n[:q]))
        res["rows"].append({"queries_per_node": ratio, "q": q, "rmq_ms": _median_ms(rmq), "inlabel_ms": _median_ms(inl),
                            "naive_ms": _median_ms(naive)})
    res["answers_identical"] = agree
    return res


def batch_size_sweep(n, dev, small=False):
    """Queries answered in batches of a given size, one launch per batch, on one preprocessed shallow
    tree (the experiment of Sec. 3.3, "Batch Size"): query throughput against batch size."""
    import torch

    import paper_2103_15217_gb300 as etl
    import synth
    P = torch.from_numpy(synth.tree_parent(n, None, seed=5)).to(dev)
    q = n
    u, v = synth.lca_queries(n, q, seed=5)
    U, V = torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev)
    h = etl.lca_preprocess(P, methods=("rmq", "inlabel"))
    out_r = torch.empty_like(U)
    out_i = torch.empty_like(U)
    ref = h.query(U, V)
    rows = []
    agree = True
    for lb in range(8 if small else 10, int(np.log2(q)) + 1, 2):
        b = 1 << lb

        def run(fn, out):
            for s in range(0, q, b):
                fn(U[s:s + b], V[s:s + b], out=out[s:s + b])
        t_r = _median_ms(lambda: run(h.query, out_r))
        t_i = _median_ms(lambda: run(h.query_inlabel, out_i))
        agree = agree and bool(torch.equal(out_r, ref) and torch.equal(out_i, ref))
        # the same launches captured once as a CUDA graph: no host work per batch
        out_r.zero_()
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=cs):
            run(h.query, out_r)
        torch.cuda.synchronize()
        t_g = _median_ms(g.replay)
        agree = agree and bool(torch.equal(out_r, ref))
        del g
        rows.append({"batch": b, "launches": (q + b - 1) // b, "rmq_ms": t_r, "rmq_queries_per_s": q / t_r * 1e3,
                     "inlabel_ms": t_i, "inlabel_queries_per_s": q / t_i * 1e3,
                     "rmq_graph_ms": t_g, "rmq_graph_queries_per_s": q / t_g * 1e3})
    h.free()
    return {"n": n, "q": q, "rows": rows, "answers_identical": agree}


# ------------------------------------------------------------------ serving

def make_serving_inputs(small: bool, seed: int = 1, nreq: int = 600):
    import synth
    from paper_2103_15217_gb300.serve import Request
    from synth.generators import make_graph
    if small:
        trees, descs = synth.serving_stream(seed=seed, nrequests=60, ntrees=8, tree_exp=(10, 13), batch_exp=(4, 12),
                                            graph_exp=(10, 12))
    else:
        trees, descs = synth.serving_stream(seed=seed, nrequests=nreq)
    parents = [synth.tree_parent(d["n"], d["grasp"], seed=d["seed"]) for d in trees]
    reqs = []
    for i, d in enumerate(descs):
        if d["kind"] == "lca":
            u, v = synth.lca_queries(trees[d["tree"]]["n"], d["q"], seed=d["seed"])
            reqs.append(Request("lca", d["t"], tree=d["tree"], u=u, v=v, rid=i))
        else:
            e = make_graph(dict(kind=d["graph"], n=d["n"], m=d["m"], seed=d["seed"]))
            reqs.append(Request("bridges", d["t"], n=d["n"], edges=e, rid=i))
    return parents, reqs


def run_serve(args):
    """Poisson stream over resident trees: continuous batching vs plain per-request launches."""
    import torch

    from paper_2103_15217_gb300.serve import Server, summarize
    parents, reqs = make_serving_inputs(args.small)
    srv = Server(parents, budget_bytes=40 << 30, slots=4)
    # offered load: scale arrival times so the stream runs at a multiple of the measured capacity
    base = [r.t for r in reqs]
    warm = srv.serve(reqs[: min(40, len(reqs))], batching=True, realtime=False)
    offline = srv.serve(reqs, batching=True, realtime=False)
    cap = summarize(offline)
    span = max(base) - min(base)
    out = {"workload": (f"{len(parents)} resident trees n log-uniform 2^10..2^22; {len(reqs)} requests, Poisson "
                        f"arrivals; LCA batches log-uniform 2^4..2^20 queries; 10% bridge requests on fresh graphs "
                        f"n log-uniform 2^10..2^22, m = 4n, easy/hard; 40 GB budget, 4 slots"),
           "capacity_units_per_s": cap["throughput"], "loads": {}}
    units = sum(r.units() for r in reqs)
    for load in (0.5, 0.8, 1.0, 1.2):
        target = units / (cap["throughput"] * load)
        for r, t in zip(reqs, base):
            r.t = (t - min(base)) / span * target
        res_b = srv.serve(reqs, batching=True)
        res_p = srv.serve(reqs, batching=False)
        same = all((a.out == b.out).all() for a, b in zip(res_b, res_p))
        out["loads"][str(load)] = {"continuous_batching": summarize(res_b), "per_request": summarize(res_p),
                                   "results_identical": bool(same)}
    for r, t in zip(reqs, base):
        r.t = t
    srv.close()
    del warm
    torch.cuda.synchronize()
    return out


# ------------------------------------------------------------------ CPU oracle arm

def run_oracle_on(trees, graphs, parts=None):
    """The oracle's fast exact paths on instances of the step's workload (all of them, or the listed
    indices into trees + graphs): Euler tour + Tarjan offline LCA per tree, DFS low-link bridges per
    graph. Returns (units, seconds)."""
    import oracle
    items = [("tree", t) for t in trees] + [("graph", g) for g in graphs]
    if parts is not None:
        items = [items[i] for i in parts]
    units, dt = 0, 0.0
    for kind, x in items:
        t0 = time.perf_counter()
        if kind == "tree":
            oracle.tree_tour(x["parent"])
            oracle.lca_offline(x["parent"], x["u"], x["v"])
            units += x["u"].shape[0]
        else:
            oracle.bridges_dfs(x["n"], x["edges"])
            units += x["edges"].shape[0]
        dt += time.perf_counter() - t0
    return units, dt


def host_cpu() -> str:
    """The host CPU as the kernel reports it (model name on x86, implementer / part on Arm)."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    if fields.get("CPU part"):
        return f"{platform.machine()} implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return platform.machine()


def cpu_baseline(trees, graphs):
    """The single-threaded oracle, timed once over the whole workload of one step (the same inputs
    the GPU line is measured on)."""
    units, dt = run_oracle_on(trees, graphs)
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one full step of the benchmark workload: " + WORKLOAD, "seconds": dt,
            "host_cores_available": os.cpu_count(), "host_cpu": host_cpu()}


def run_reference(args):
    """The reference arm: the CPU oracle on the benchmark's own inputs. Each step is one instance of
    the five (three trees, two graphs) in rotation, so K steps cover the workload K / 5 times and
    the run stays within minutes; value = units / time over the K timed steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    trees, graphs = make_inputs(args.small, seed=replica_seed(0, args.seed))
    ninst = len(trees) + len(graphs)
    for i in range(args.warmup):
        run_oracle_on(trees, graphs, [i % ninst])
    tot_units, tot_t = 0, 0.0
    for i in range(args.steps):
        u, t = run_oracle_on(trees, graphs, [i % ninst])
        tot_units += u
        tot_t += t
    value = tot_units / tot_t
    sample = (f"one instance of the workload per step, the {ninst} instances in rotation "
              f"({args.steps} steps): " + (WORKLOAD if not args.small else "small functional check"))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD if not args.small else "small functional check", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host_cores_available": os.cpu_count(), "host_cpu": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_case(args):
    """One workload, run twice (the second run is the one to capture)."""
    import torch

    import paper_2103_15217_gb300 as etl
    import synth
    etl.build()
    dev = torch.device("cuda", 0)
    n = args.n
    if args.case in ("batch_trees", "batch_graphs"):
        B = make_batch_inputs(small=False)
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        for _ in range(2):
            if args.case == "batch_trees":
                h = etl.lca_preprocess_batch(T(np.concatenate(B["tp"])), T(B["toff"]), max(d["n"] for d in B["trees"]))
                h.query_batch(T(np.concatenate(B["ti"])), T(np.concatenate(B["tu"])), T(np.concatenate(B["tv"])))
                h.free()
            else:
                etl.find_bridges_batch(T(np.concatenate(B["ge"])), T(B["eoff"]), T(B["noff"]), int(B["noff"][-1]))
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "launches": etl.launch_count()}))
        return
    if args.case == "lca":
        parent = torch.from_numpy(synth.tree_parent(n, args.grasp or None, seed=1)).to(dev)
        u, v = (torch.from_numpy(x).to(dev) for x in synth.lca_queries(n, n, seed=1))
        for _ in range(2):
            h = etl.lca_preprocess(parent)
            h.query(u, v)
            h.free()
    else:
        m = 8 * n if args.case == "easy" else 5 * n
        e = synth.easy_graph(n, m, seed=1) if args.case == "easy" else synth.hard_graph(n, m - (n - 1), n // 64, seed=1)
        edges = torch.from_numpy(e).to(dev)
        for _ in range(2):
            etl.find_bridges(edges, n)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": n, "launches": etl.launch_count()}))


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
