#!/usr/bin/env python3
"""Benchmark: k-bisimulation refinement on the 16M-node / 256M-edge graph.

One step = one full pass of the hot path on a device-resident graph: level 0
(label grouping) and refinement rounds 1..k (k = 10) until the block count
stops changing.  Metric: edge-rounds per second = E x rounds run / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank refines its
own replica of the graph; there is no data-path collective ("replicas only":
the single-graph path does not shard) and value = N x E x rounds / max time.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edge-rounds/sec (k-bisimulation refinement, 1 GB300)"
UNIT = "edge-rounds/s"
K_ROUNDS = 10
L2_BYTES = 129 * 1024 * 1024

# Algorithmic bytes of one refinement round (implementation-independent):
# per edge: read dst + label (5 B), write its distinct key (8 B), read that key
# once for the exact comparison (8 B) = 21 B; per node: offsets 8, pId_{i-1} 4,
# hash write 8, one read + write of a 16 B grouping record 32, pId_i write 4 = 56 B.
BYTES_PER_EDGE = 21
BYTES_PER_NODE = 56
# Split of those bytes over the kernel classes the library times, as
# (bytes per edge, bytes per node) of the edges and nodes each class covers:
#   signature kernels: 13 B/edge + 20 B/node (dst+label read, key write;
#   offsets, pId_{i-1}, hash write), grouping: 16 B/node, verification:
#   16 B/node, renumbering: 4 B/node.  The formula's 8 B/edge read of the keys
#   for the exact comparison is charged to no class: verification compares only
#   the nodes that share their previous block with another node (Proposition 1
#   keeps the others alone), so how many keys it reads depends on the graph,
#   and the per-class fractions are lower bounds on the work each class does.
KERNEL_BYTES = {
    "sig_small": (13, 20),
    "sig_medium": (13, 20),
    "sig_hub": (13, 20),
    "group": (0, 16),
    "verify": (0, 16),
    "renumber": (0, 4),
}
# Out-degree ranges of the signature kernel classes (the library's split).
SIG_DEGREES = {"sig_small": (0, 64), "sig_medium": (65, 4096), "sig_hub": (4097, None)}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_powerlaw_4m_64m.json")


def class_units(g):
    """(edges, nodes) each kernel class processes per round."""
    d = np.diff(g.offsets.astype(np.int64))
    out = {}
    for k, (lo, hi) in SIG_DEGREES.items():
        m = (d >= lo) & (d <= hi) if hi is not None else (d >= lo)
        out[k] = (int(d[m].sum()), int(m.sum()))
    for k in ("group", "verify", "renumber"):
        out[k] = (g.num_edges, g.num_nodes)
    return out


def recorded_traffic(cls, units):
    """DRAM bytes per round of a kernel class from the committed ncu summary, if it
    was taken on the current kernel sources.  The capture is of the same
    generator at a smaller scale (4M nodes / 64M edges: inputs larger than L2,
    a few GB on the device), which records the units each class processed
    there; the traffic is scaled by this workload's units over those (edges for
    the signature classes, nodes for the per-node classes).  `units`: this
    workload's (edges, nodes) of the class."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    from ncu_summary import source_digest
    if t.get("source_sha256") != source_digest():
        return None
    v = t.get("dram_bytes_per_round", {}).get(cls)
    cu = t.get("class_units", {}).get(cls)
    if v is None or not cu:
        return None
    if cls.startswith("sig"):
        return float(v) * units[0] / max(cu["edges"], 1)
    return float(v) * units[1] / max(cu["nodes"], 1)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = 16M/256M)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--skip-clocks", action="store_true")
    p.add_argument("--hub-bucket-keys", type=int, default=0, choices=[0, 2048, 4096, 8192],
                   help="hub bucket size (0 = tuned by the library on the first refinement)")
    p.add_argument("--workload", default="single", choices=["single", "batched", "large", "serve", "update"],
                   help="single: the 16M/256M graph (the headline line); batched: 4096 graphs "
                        "(times --scale) in one batched build vs one build per graph; large: the "
                        "256M-node / 2B-edge graph; serve: 64 resident graphs under Poisson request "
                        "streams; update: maintenance batches on the 16M/256M graph, incremental "
                        "against recomputation")
    p.add_argument("--batch", type=int, default=1000, help="edges per maintenance batch (update)")
    p.add_argument("--graph", default="powerlaw", choices=["powerlaw", "uniform"],
                   help="update: the 16M/256M power-law graph, or a 6.4M-node / 64M-edge graph with the "
                        "100K/1M generator's distributions (uniform targets), the largest serving graph")
    p.add_argument("--k", type=int, default=3, help="levels kept by maintenance (update)")
    p.add_argument("--requests", type=int, default=120, help="requests per arrival rate (serve)")
    return p.parse_args()


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks of the job (x itself with one rank); the
    reduction runs on the device for NCCL, on the host for gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank (weak scaling),
    the job takes as long as its slowest rank."""
    return world * units_per_rank / (ms_max / 1000.0)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, enabled=True):
        self.proc = None
        self.path = None
        self.device_index = device_index
        if not enabled:
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def workload(scale, kind="single"):
    from paper_1210_0748_gb300 import synth
    if kind == "large":
        g = synth.config_large_single(scale=scale)
        return g, {"workload": "powerlaw graph: %d nodes, %d edges, out-degree Pareto alpha=2.0 (hubs to 1M), "
                               "preferential-attachment targets, 64 node labels and 16 edge labels Zipf(1.3), "
                               "k=10 with early stop" % (g.num_nodes, g.num_edges),
                   "nodes": g.num_nodes, "edges": g.num_edges, "k": K_ROUNDS,
                   "l2": "inputs larger than L2 (no flush needed)"}
    g = synth.config_single_large(scale=scale)
    return g, {"workload": "powerlaw graph: %d nodes, %d edges, out-degree Pareto alpha=2.1 (hubs "
                           "to 1M), preferential-attachment targets, 16 node labels Zipf(1.2), "
                           "32 edge labels Zipf(1.5), k=10 with early stop" % (g.num_nodes, g.num_edges),
               "nodes": g.num_nodes, "edges": g.num_edges, "k": K_ROUNDS,
               "l2": "inputs larger than L2 (no flush needed)"}


def cpu_baseline(scale_full):
    """The oracle as it stands, single-threaded, on a bounded sample: the same
    generator at 1/16 of the size (1M nodes, 16M edges), k = 10."""
    import oracle
    from paper_1210_0748_gb300 import synth
    sc = scale_full / 16.0
    g = synth.config_single_large(scale=sc)
    src = g.src()
    r = oracle.kbisim(g.num_nodes, g.node_label, src, g.dst, g.edge_label, K_ROUNDS)
    secs = float(np.sum(r.round_seconds))
    return {"value": g.num_edges * r.rounds_run / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "a 1/16 sample, not the benchmark graph: the same generator at %d nodes / %d "
                      "edges, k=10 with early stop (%d rounds, %.1f s of rounds); the value is this "
                      "sample's edges x rounds / oracle round time" % (g.num_nodes, g.num_edges,
                                                                     r.rounds_run, secs)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1210_0748_gb300 import synth
    _, cfg = workload(args.scale)
    sc = args.scale / 64.0  # bounded sample per step: 250K nodes, 4M edges
    g = synth.config_single_large(scale=sc)
    src = g.src()
    for _ in range(args.warmup):
        oracle.kbisim(g.num_nodes, g.node_label, src, g.dst, g.edge_label, K_ROUNDS)
    t0 = time.perf_counter()
    rounds = 0
    for _ in range(args.steps):
        r = oracle.kbisim(g.num_nodes, g.node_label, src, g.dst, g.edge_label, K_ROUNDS)
        rounds += r.rounds_run
    dt = time.perf_counter() - t0
    value = g.num_edges * rounds / dt
    sample = ("a 1/64 sample per step, not the benchmark graph: the oracle on the same generator "
              "at %d nodes / %d edges, k=10 with early stop; the value is this sample's edges x "
              "rounds / time" % (g.num_nodes, g.num_edges))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": cfg,
            "sample": {"nodes": g.num_nodes, "edges": g.num_edges,
                       "note": "each step times the oracle on this sample of the workload named in "
                               "config (the full graph takes about a minute per build on one core)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """Many independent graphs: one kbisim_build_many against one kbisim_build
    per graph, inputs resident on the device for both, each arm timed over
    whole builds (load, refinement, per-graph results) with the host work
    that a build needs.  Value: sum over graphs of edges x rounds computed,
    per second."""
    import torch
    from types import SimpleNamespace
    from paper_1210_0748_gb300 import synth
    from paper_1210_0748_gb300.kbisim import KBisim, concat_graphs
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    count = max(1, int(round(4096 * args.scale)))
    graphs, ks = synth.config_batched(count=count)
    union, starts = concat_graphs(graphs)

    def on_dev(g):
        return SimpleNamespace(num_nodes=g.num_nodes,
                               offsets=torch.from_numpy(g.offsets.view(np.int64)).to(dev),
                               dst=torch.from_numpy(g.dst.view(np.int32)).to(dev),
                               edge_label=torch.from_numpy(g.edge_label).to(dev),
                               node_label=torch.from_numpy(g.node_label.view(np.int32)).to(dev))

    U = on_dev(union)
    solo = [on_dev(g) for g in graphs]
    stream = torch.cuda.Stream(device=local_rank)
    kb = KBisim(device=local_rank, stream=stream)
    for _ in range(max(1, args.warmup)):
        kb.build_many(None, ks, union=(U, starts))
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        kb.build_many(None, ks, union=(U, starts))
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / steps
    rounds = [kb.many_info(j)[0] for j in range(count)]
    work = float(sum(g.num_edges * r for g, r in zip(graphs, rounds)))
    for j in range(min(count, 8)):  # warm-up of the solo path
        kb.build(None, ks[j], num_nodes=solo[j].num_nodes, node_label=solo[j].node_label, dst=solo[j].dst,
                 edge_label=solo[j].edge_label, offsets=solo[j].offsets)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solo_rounds = []
    for j, g in enumerate(solo):
        r = kb.build(None, ks[j], num_nodes=g.num_nodes, node_label=g.node_label, dst=g.dst,
                     edge_label=g.edge_label, offsets=g.offsets)
        solo_rounds.append(r.rounds_run)
    torch.cuda.synchronize()
    t_solo = time.perf_counter() - t0
    assert solo_rounds == rounds, "batched and solo builds ran different rounds"
    kb.close()
    line = {"metric": "edge-rounds/sec, batched build of %d graphs (1 GB300)" % count,
            "value": work / t_batch, "unit": "edge-rounds/s", "n_gpus": 1, "steps": steps,
            "warmup": max(1, args.warmup), "ms_per_step": 1000 * t_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "%d graphs, edges log-uniform in [1K, 1M], nodes = edges/8, out-degree "
                                   "Zipf(2.0) capped at 10K, uniform targets, 8 node / 4 edge labels uniform, "
                                   "k uniform in 1..10" % count,
                       "graphs": count, "edges": int(union.num_edges), "nodes": int(union.num_nodes)},
            "one_at_a_time": {"value": work / t_solo, "unit": "edge-rounds/s", "ms_total": 1000 * t_solo},
            "speedup_vs_one_at_a_time": t_solo / t_batch,
            "timing": "host wall clock around whole builds with CUDA synchronisation (both arms)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_update(args):
    """Maintenance batches (half inserts of random edges, half deletions of
    stored edges) on the 16M/256M graph (or the uniform 6.4M/64M one) with k
    levels: the same sequence of batches through the library's timed choice of
    path (options.maintain = 1, the default: the value of the line), through
    the frontier path whenever it applies (maintain = 2) and through
    recomputation (maintain = 0), each timed per update (host wall clock around
    kbisim_update, which waits for its stream), with the levels of all handles
    compared after every batch."""
    import torch
    from paper_1210_0748_gb300.kbisim import KBisim
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if args.graph == "uniform":
        from paper_1210_0748_gb300 import synth
        m = int(64_000_000 * args.scale)
        g = synth.uniform_zipf_graph(m // 10, m, zipf_s=2.0, dmax=10_000, node_labels=8, edge_labels=4)
        cfg = {"workload": "graph of %d nodes, %d edges: out-degree Zipf(2.0) capped at 10K, uniform targets, "
                           "8 node labels and 4 edge labels uniform" % (g.num_nodes, g.num_edges),
               "nodes": g.num_nodes, "edges": g.num_edges}
        n_labels = 4
    else:
        g, cfg = workload(args.scale)
        n_labels = 32
    rng = np.random.default_rng(77)
    src = g.src()
    nb = max(2, args.batch)
    batches = []
    for _ in range(args.warmup + args.steps):
        ni, nd = nb // 2, nb - nb // 2
        ins = (rng.integers(0, g.num_nodes, ni).astype(np.uint32), rng.integers(0, g.num_nodes, ni).astype(np.uint32),
               rng.integers(0, n_labels, ni).astype(np.uint32))
        e = rng.integers(0, g.num_edges, nd)
        dels = (src[e], g.dst[e], g.edge_label[e].astype(np.uint32))
        batches.append((ins, dels))
    out = {}
    levels = {}
    for name, maintain in (("timed", True), ("incremental", "always"), ("recompute", False)):
        stream = torch.cuda.Stream(device=local_rank)
        kb = KBisim(device=local_rank, stream=stream, maintain=maintain)
        kb.build(g, args.k)
        times, paths, nodes = [], [], []
        for i, (ins, dels) in enumerate(batches):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            kb.update(args.k, ins=ins, dels=dels)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt * 1000.0)
                info = kb.update_info()
                paths.append(info["reason"])
                nodes.append(info["frontier_nodes"])
            levels.setdefault(i, []).append(kb.pids(args.k))
        out[name] = {"ms_per_update_median": float(np.median(times)), "ms_per_update_mean": float(np.mean(times)),
                     "paths": {p: paths.count(p) for p in set(paths)},
                     "frontier_nodes_median": float(np.median(nodes)) if nodes else 0.0}
        kb.close()
    same = all(np.array_equal(v[0], x) for v in levels.values() for x in v[1:])
    line = {"metric": "maintenance: ms per update batch of %d edges, k=%d (1 GB300)" % (nb, args.k),
            "value": out["timed"]["ms_per_update_median"], "unit": "ms", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(cfg, batch_edges=nb, k=args.k),
            "timed": out["timed"], "incremental": out["incremental"], "recompute": out["recompute"],
            "speedup": out["recompute"]["ms_per_update_median"] / out["timed"]["ms_per_update_median"],
            "speedup_incremental": out["recompute"]["ms_per_update_median"] / out["incremental"]["ms_per_update_median"],
            "levels_equal": same,
            "timing": "host wall clock around each kbisim_update (the call waits for its stream)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0 if same else 1


def run_serve(args):
    """Resident graphs under Poisson request streams (70% update batches of
    1K..1M edges, 30% rebuilds at k 3..10) at several arrival rates: latency
    percentiles from arrival to result, and throughput."""
    import torch
    from paper_1210_0748_gb300 import synth
    from paper_1210_0748_gb300.serve import Server, make_requests
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    graphs, ks = synth.config_serving(scale=args.scale)
    srv = Server(graphs, ks, slots=8, device=local_rank)
    warm = make_requests(graphs, rate=0.0, count=16, seed=99)
    srv.serve(warm, realtime=False)
    runs = []
    for i, rate in enumerate([10.0, 100.0, 1000.0]):
        reqs = make_requests(graphs, rate=rate, count=args.requests, seed=1 + i)
        t0 = time.perf_counter()
        out = srv.serve(reqs, realtime=True)
        span = time.perf_counter() - t0
        lat = np.array([o.latency for o in out]) * 1000.0
        work = float(sum(o.edges * o.rounds_run for o in out))
        runs.append({"rate_per_s": rate, "requests": len(out), "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "throughput_req_per_s": len(out) / span,
                     "edge_rounds_per_s": work / span,
                     "updates": sum(o.kind == "update" for o in out)})
    # the saturated stream again with one request at a time: what overlap buys
    srv.slots = 1
    reqs = make_requests(graphs, rate=1000.0, count=args.requests, seed=3)
    t0 = time.perf_counter()
    out = srv.serve(reqs, realtime=True)
    span1 = time.perf_counter() - t0
    one_at_a_time = {"throughput_req_per_s": len(out) / span1,
                     "p50_ms": float(np.percentile([o.latency * 1000 for o in out], 50)),
                     "p99_ms": float(np.percentile([o.latency * 1000 for o in out], 99))}
    srv.close()
    best = max(runs, key=lambda r: r["throughput_req_per_s"])
    line = {"metric": "serving: requests/s with p50/p99 latency (1 GB300)", "value": best["throughput_req_per_s"],
            "unit": "requests/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "%d resident graphs, edges log-uniform in [1M, 64M] x %g, nodes = edges/10, "
                                   "100K/1M-generator distributions; Poisson arrivals, 70%% update batches of "
                                   "1K..1M edges (half inserts, half deletes of generated edges), 30%% rebuilds "
                                   "at k 3..10; 8 slots" % (len(graphs), args.scale),
                       "graphs": len(graphs), "edges": int(sum(g.num_edges for g in graphs))},
            "rates": runs, "one_slot_at_1000_per_s": one_at_a_time,
            "overlap_speedup": runs[-1]["throughput_req_per_s"] / one_at_a_time["throughput_req_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world = dist_env()[2]
    if args.gpus != world:
        print("bench.py: --gpus %d but WORLD_SIZE=%d; launch N > 1 ranks with torch.distributed.run "
              "(one process per GPU)" % (args.gpus, world), file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "update":
        return run_update(args)
    import torch
    from paper_1210_0748_gb300.kbisim import KBisim

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    g, cfg = workload(args.scale, args.workload)
    if args.workload == "large":  # a parity-scale case: no host-buffer leg, no CPU sample
        args.no_e2e = True
        args.no_cpu_baseline = True
    E, N = g.num_edges, g.num_nodes
    stream = torch.cuda.Stream(device=local_rank)
    kb = KBisim(device=local_rank, stream=stream, collect_timing=True, hub_bucket_keys=args.hub_bucket_keys)
    kb.load(g)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        res = kb.refine(K_ROUNDS)
    torch.cuda.synchronize()
    kb.reset_times()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank, enabled=not args.skip_clocks)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rounds = 0
    for _ in range(args.steps):
        res = kb.refine(K_ROUNDS)
        rounds += res.rounds_run
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ktimes = kb.kernel_times()
    barrier()
    ms_max = max_over_ranks(ms_total)
    ms_step = ms_max / args.steps
    value = job_value(E * rounds, world, ms_max)

    # roofline: the whole refinement round against the fixed algorithmic bytes,
    # and each kernel class against its share of those bytes (per call of the
    # class: once per round for the signature classes, once per level -- level
    # 0 included -- for grouping, verification and renumbering)
    peak, peak_kind = load_peaks()
    rounds_per_step = rounds / args.steps
    gpu_launches = int(sum(c for _, c in ktimes.values()))
    round_ms = (ms_total / args.steps - ktimes["label_group"][0] / args.steps) / max(rounds_per_step, 1)
    round_bytes = BYTES_PER_EDGE * E + BYTES_PER_NODE * N
    units = class_units(g)
    per_class = {}
    for cls, (be, bn) in KERNEL_BYTES.items():
        calls = rounds if cls.startswith("sig") else rounds + args.steps
        ms, launches = ktimes[cls]
        if calls == 0 or ms <= 0:
            continue
        e_c, n_c = units[cls]
        byts = be * e_c + bn * n_c
        ms_call = ms / calls
        per_class[cls] = {"achieved": byts / (ms_call / 1000.0) / 1e9, "frac": byts / (ms_call / 1000.0) / 1e9 / peak,
                          "algorithmic_bytes_per_call": byts, "ms_per_call": ms_call,
                          "launches_per_call": launches / calls, "edges": e_c, "nodes": n_c}
    dom = max(per_class, key=lambda c: ktimes[c][0])
    d = per_class[dom]
    # measured DRAM bytes of the class per round (ncu), per launch like the algorithmic bytes
    traffic_round = recorded_traffic(dom, units[dom]) if args.workload == "single" else None
    traffic = traffic_round / d["launches_per_call"] if traffic_round is not None else None
    names = {"sig_small": "k_sig_small (out-degree <= 64, one thread per node)",
             "sig_medium": "k_sig_chunk (out-degree 65..4096, CTA chunks)",
             "sig_hub": "k_hub_sample, k_hub_chunk or k_hub_scatter per hub, k_hub_bucket, k_hub_finish (out-degree > 4096)",
             "group": "k_group_insert", "verify": "k_group_verify", "renumber": "renumbering kernels"}
    roofline = {"bound": "hbm", "kernel": names.get(dom, dom), "achieved": d["achieved"], "peak": peak,
                "unit": "GB/s", "frac": d["frac"], "peak_kind": peak_kind, "traffic": traffic,
                "traffic_per_round": traffic_round, "algorithmic_bytes_per_round": d["algorithmic_bytes_per_call"],
                "algorithmic_bytes_per_launch": d["algorithmic_bytes_per_call"] / d["launches_per_call"],
                "avg_launch_ms": d["ms_per_call"] / d["launches_per_call"],
                "launches_per_round": d["launches_per_call"]}
    round_achieved = round_bytes / (round_ms / 1000.0) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": cfg, "rounds_per_step": rounds_per_step, "roofline": roofline,
            "round_roofline": {"achieved": round_achieved, "peak": peak, "unit": "GB/s",
                               "frac": round_achieved / peak, "avg_round_ms": round_ms,
                               "algorithmic_bytes": round_bytes},
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in ktimes.items()},
            "kernel_roofline": {k: {"achieved": v["achieved"], "frac": v["frac"], "ms_per_call": v["ms_per_call"]}
                                for k, v in per_class.items()},
            "hub_bucket_keys": kb.hub_bucket_keys, "gpu_launches": gpu_launches, "clocks": clk}

    # end to end through the public API: pinned host inputs -> build -> level k to host
    if not args.no_e2e:
        pin = {"offsets": torch.from_numpy(g.offsets.view(np.int64)).pin_memory(),
               "dst": torch.from_numpy(g.dst.view(np.int32)).pin_memory(),
               "edge_label": torch.from_numpy(g.edge_label).pin_memory(),
               "node_label": torch.from_numpy(g.node_label.view(np.int32)).pin_memory()}
        host_g = type(g)(N, pin["offsets"].numpy().view(np.uint64), pin["dst"].numpy().view(np.uint32),
                         pin["edge_label"].numpy(), pin["node_label"].numpy().view(np.uint32))
        out = torch.empty(N, dtype=torch.int32).pin_memory()
        out_np = out.numpy()
        kb2 = KBisim(device=local_rank, stream=stream)
        r0 = kb2.build(host_g, K_ROUNDS)  # warm-up
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e2e_rounds = 0
        e2e_steps = max(1, min(args.steps, 10))
        marks = [t0]
        for _ in range(e2e_steps):
            r = kb2.build(host_g, K_ROUNDS)  # returns once the counts are on the host
            kb2._check(kb2._lib.kbisim_pids(kb2._h, K_ROUNDS, out_np.ctypes.data, 0))
            e2e_rounds += r.rounds_run
            marks.append(time.perf_counter())
        dt = max_over_ranks(time.perf_counter() - t0)
        h2d = sum(v.numel() * v.element_size() for v in pin.values())
        per_build = np.diff(np.array(marks)) * 1000.0
        line["e2e"] = {"value": job_value(E * e2e_rounds, world, dt * 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": N * 4 + 8 * (K_ROUNDS + 1),
                       "ms_per_step": 1000 * dt / e2e_steps,
                       "ms_per_build": {"min": float(per_build.min()), "median": float(np.median(per_build)),
                                        "max": float(per_build.max())}}
        # where a build's time goes: three more builds, each phase timed on its own
        # (outside the timed region above)
        phases = {"load": [], "refine": [], "pids_to_host": []}
        for _ in range(3):
            a0 = time.perf_counter()
            kb2.load(host_g)
            torch.cuda.synchronize(local_rank)
            a1 = time.perf_counter()
            kb2.refine(K_ROUNDS)
            torch.cuda.synchronize(local_rank)
            a2 = time.perf_counter()
            kb2._check(kb2._lib.kbisim_pids(kb2._h, K_ROUNDS, out_np.ctypes.data, 0))
            a3 = time.perf_counter()
            phases["load"].append(a1 - a0)
            phases["refine"].append(a2 - a1)
            phases["pids_to_host"].append(a3 - a2)
        line["e2e"]["phase_ms_median"] = {k: 1000.0 * float(np.median(v)) for k, v in phases.items()}
        kb2.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.scale)
    kb.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
