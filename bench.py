#!/usr/bin/env python
"""Benchmark: exact minimum vertex cover on one GB300 per rank.

Workload (one step = one exact MVC solve through the C ABI, root reduction,
induced subgraph, search and witness included):
    Chung-Lu power-law graph, n = 50,000, exponent 2.5, mean degree 6,
    maximum degree 2,000, int32 CSR, seed 1000 + rank (synthetic; the paper's
    datasets are not available).

value   graphs/s over all ranks, CSR already resident in HBM, L2 flushed
        (256 MiB write) before every timed step
e2e     the same metric through vc_load_csr from pinned host memory, the
        solve, and the cover read back to the host, every step
roofline of the dominant kernel (root reduction), achieved algorithmic bytes
        per launch / its CUDA-event duration vs the measured HBM copy peak
cpu_baseline  the CPU oracle (sequential Algorithm 2 in C) on the same graph

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402

METRIC = "graphs/sec & search-tree nodes/sec at exact MVC; p99 latency; batched vs plain"
WORKLOADS = {
    # the headline: plain exact MVC of one Chung-Lu power-law graph
    "chung_lu_50k": dict(workload="chung_lu_50k", n=50_000, gamma=2.5, avg_deg=6.0, max_deg=2000.0),
    # search-dominated: 8 copies of G(48, 0.12) hung on a 2-vertex chain
    "component_heavy_8x48": dict(workload="component_heavy_8x48", copies=8, copy_n=48, p=0.12, chain=2),
}
WORKLOAD = WORKLOADS["chung_lu_50k"]
L2_FLUSH_BYTES = 256 << 20


def make_graph(rank: int):
    w = WORKLOAD
    if w["workload"] == "chung_lu_50k":
        return gg.chung_lu(w["n"], w["gamma"], w["avg_deg"], w["max_deg"], 1000 + rank)
    return gg.component_heavy(1 + rank, copies=w["copies"], copy_n=w["copy_n"], p=w["p"], chain=w["chain"])


def solve_options():
    """Search capacities: the defaults, or modest fixed ones for the
    search-dominated workload (keeps its device footprint small)."""
    if WORKLOAD["workload"] == "component_heavy_8x48":
        return dict(stack_depth=128, registry_capacity=1 << 18)
    return {}


def kernel_traffic(kernel: str, workload: str | None = None):
    """DRAM bytes per launch from the committed ncu summary, when it was taken
    on the current source of that kernel (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[workload or WORKLOAD["workload"]]
    except Exception:
        return None
    if rec.get("kernel") != kernel:
        return None
    src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    return rec["traffic"] if hashlib.sha256(src).hexdigest() == rec["sha256"] else None


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def combine_over_ranks(local_ms: float, steps: int, world: int):
    """Replicas: the timed region is the slowest rank's (MAX over ranks) and
    the value counts the graphs of every rank: (max_ms, world * steps / max_s).
    Uses the default process group when world > 1 (a CUDA tensor under NCCL,
    a CPU tensor under gloo)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(local_ms)], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    return local_ms, world * steps / (local_ms / 1e3)


def shard_by_cost(costs, world: int):
    """Split independent graphs over `world` ranks: longest first, each to
    the rank with the least cost so far (LPT).  Returns one ascending index
    list per rank; every index appears exactly once."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def host_group():
    """A gloo process group over every rank, for the host-side gathers of
    the sharded batch (no device collective on the data path)."""
    import torch.distributed as dist
    return dist.new_group(backend="gloo")


def combine_search(local: dict, world: int, group=None) -> dict:
    """Sharded batch: every rank solved its share; the job's time is the
    slowest rank's, its queries and nodes those of every rank."""
    if world == 1:
        return local
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, {k: local[k] for k in ("queries", "nodes", "ms_wall", "ms_kernel", "wrong",
                                                          "over", "bytes")}, group=group)
    ms_wall = max(p["ms_wall"] for p in parts)
    ms_kernel = max(p["ms_kernel"] for p in parts)
    out = dict(local)
    for k in ("queries", "nodes", "wrong", "over", "bytes"):
        out[k] = sum(p[k] for p in parts)
    out["ms_wall"], out["ms_kernel"] = ms_wall, ms_kernel
    out["per_rank_queries"] = [p["queries"] for p in parts]
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm

def cpu_oracle_run(steps: int, warmup: int):
    """The oracle as it stands, on this host: one workload graph per step."""
    import oracle
    oracle.build()
    g = make_graph(0)
    for _ in range(warmup):
        oracle.mvc(g.n, g.row_ptr, g.col)
    t0 = time.perf_counter()
    size = None
    for _ in range(steps):
        size = oracle.mvc(g.n, g.row_ptr, g.col)[0]
    dt = time.perf_counter() - t0
    return steps / dt, dt / steps * 1e3, size


def host_cpu() -> dict:
    """The host's core count and CPU model, for the CPU baselines."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count() or 1, "model": model}


def cpu_oracle_all_cores(jobs, budget: int = 0, max_s: float = 15.0) -> dict:
    """The oracle over independent graphs on every host core.  jobs: a list
    of (graph, k) with k < 0 for a minimum cover.  Threads suffice: the
    oracle is reentrant C and ctypes releases the GIL during the call.  Jobs
    are taken in order, a core-count wave at a time, until max_s has passed
    (a bounded sample); returns the rate over the jobs done."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1

    def one(job):
        g, k = job
        try:
            if k < 0:
                oracle.mvc(g.n, g.row_ptr, g.col, node_budget=budget)
            else:
                oracle.pvc(g.n, g.row_ptr, g.col, k, node_budget=budget)
            return 1
        except oracle.OracleBudgetExceeded:
            return 0

    done = over = 0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        for i in range(0, len(jobs), cores):
            for r in ex.map(one, jobs[i:i + cores]):
                done += 1
                over += 1 - r
            if time.perf_counter() - t0 > max_s:
                break
    dt = time.perf_counter() - t0
    return {"per_s": round(done / dt, 1), "jobs": done, "of": len(jobs), "over_budget": over,
            "cores": cores, "s": round(dt, 3)}


def reference_main(args, rank, world):
    if rank != 0:
        return
    value, ms, size = cpu_oracle_run(args.steps, args.warmup)
    sample = (f"full {WORKLOAD['workload']} graph, {args.steps} timed solves after "
              f"{args.warmup} warm-up, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "graphs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": dict(WORKLOAD, answer=size),
        "cpu_baseline": {"value": round(value, 6), "unit": "graphs/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "graphs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line, default=_json_default), flush=True)


# ------------------------------------------------------------------ our arm

def root_algorithmic_bytes(g, st) -> int:
    """Bytes the root phase must move at least once: read the CSR, write the
    cover flags and the forced list, write the induced CSR and its id map."""
    csr = 4 * (g.n + 1) + 4 * int(g.row_ptr[-1])
    outs = g.n + 4 * st["forced"] + 4 * (st["n_induced"] + 1) + 8 * st["m_induced"] + 4 * st["n_induced"]
    return csr + outs


def extra_workloads(vc, torch, stream, peak):
    """Context numbers beside the headline: plain vs batched launches of small
    graphs, the search kernel on a component-heavy graph, and a mixed batch
    under a per-query node budget.  Each part runs for a few seconds."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        ev0.record(stream)
        r = fn()
        ev1.record(stream)
        ev1.synchronize()
        return r, ev0.elapsed_time(ev1)

    out = {}
    # G(n=80, m=200): one launch per graph vs one batched launch
    gs = [gg.gnm(80, 200, s) for s in range(256)]
    dgs = [vc.Graph.from_csr(g.row_ptr, g.col, stream=stream) for g in gs]
    for d in dgs[:8]:
        vc.solve_min(d)
    lat, nodes = [], 0
    for d in dgs:
        (size, _, st), ms = timed(lambda: vc.solve_min(d))
        lat.append(ms)
        nodes += st["nodes"]
    tuned, _, _ = vc.autotune(dgs, repeats=2)
    vc.solve_batch(dgs[:16], opts=tuned)
    (sizes, _, status, _, bst), bms = timed(lambda: vc.solve_batch(dgs, opts=tuned))
    out["gnm_80_200"] = {
        "graphs": len(dgs), "plain_graphs_per_s": round(len(dgs) / (sum(lat) / 1e3), 1),
        "plain_p50_ms": round(float(np.percentile(lat, 50)), 4), "plain_p99_ms": round(float(np.percentile(lat, 99)), 4),
        "plain_nodes_per_s": round(nodes / (sum(lat) / 1e3), 1),
        "batched_graphs_per_s": round(len(dgs) / (bms / 1e3), 1), "batched_ms": round(bms, 3),
        "batched_nodes_per_s": round(bst["nodes"] / (bms / 1e3), 1),
        "batched_options": {f: getattr(tuned, f) for f in vc.TUNED_FIELDS},
        "cpu_oracle_all_cores": cpu_oracle_all_cores([(g, -1) for g in gs])}
    for d in dgs:
        d.close()

    # component-heavy: 8 copies of G(48, 0.12) on a 2-vertex chain
    g = gg.component_heavy(1, copies=8, copy_n=48, p=0.12, chain=2)
    d = vc.Graph.from_csr(g.row_ptr, g.col, stream=stream)
    vc.solve_min(d)
    (size, _, st), ms = timed(lambda: vc.solve_min(d))
    d.close()
    gbs = st["search_bytes"] / (st["ms_search"] / 1e3) / 1e9 if st["ms_search"] > 0 else 0.0
    out["component_heavy_8x48"] = {
        "n": g.n, "answer": size, "nodes": st["nodes"], "ms_total": round(ms, 3),
        "ms_search_kernel": round(st["ms_search"], 3),
        "nodes_per_s": round(st["nodes"] / (st["ms_search"] / 1e3), 1),
        "component_branches": st["component_branches"], "workers": st["workers"], "team": st["team"],
        "search_roofline": {"bound": "hbm", "kernel": "search_kernel", "achieved": round(gbs, 3),
                            "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 6),
                            "algorithmic_bytes": st["search_bytes"],
                            "bytes_per_node": round(st["search_bytes"] / max(1, st["nodes"]), 1),
                   "crown_forced": st["crown_forced"], "crown_removed": st["crown_removed"]}}

    # mixed batch (n in [40, 400]; half G(n,p), half Chung-Lu), per-query budget
    mix = gg.batch_pvc_mix(512, 7, n_lo=40, n_hi=400)
    dms = [vc.Graph.from_csr(h.row_ptr, h.col, stream=stream) for h in mix]
    budget = 500_000
    # first pass: which queries finish within the budget (the rest are dropped)
    _, _, status, _, _ = vc.solve_batch(dms, node_budget=budget, raise_on_error=False)
    solved = [i for i in range(len(dms)) if status[i] == 0]
    keep = [dms[i] for i in solved]
    vc.solve_batch(keep[:32], raise_on_error=False)
    (sizes, _, st2, _, bst), bms = timed(lambda: vc.solve_batch(keep, node_budget=budget, raise_on_error=False))
    plain = []
    for i in solved:
        try:
            (_, _, _), ms = timed(lambda: vc.solve_min(dms[i], node_budget=budget))
        except vc.VcError:
            continue   # the search order differs between launches; rarely over budget alone
        plain.append(ms)
    out["mixed_batch_512"] = {
        "queries": len(dms), "solved": len(solved), "dropped_over_budget": int((status == vc.VC_EBUDGET).sum()),
        "node_budget_per_query": budget, "batched_ms": round(bms, 3),
        "batched_graphs_per_s": round(int((st2 == 0).sum()) / (bms / 1e3), 1),
        "plain_graphs_per_s": round(len(plain) / (sum(plain) / 1e3), 1) if plain else None,
        "batched_nodes_per_s": round(bst["nodes"] / (bms / 1e3), 1)}
    for d in dms:
        d.close()
    return out


def _log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def _json_default(o):
    """numpy scalars in the JSON line."""
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(f"not JSON serializable: {type(o).__name__}")


def cover_ok(g, cover) -> bool:
    """Every edge has an end in the cover (a plain edge check, no solver)."""
    flags = np.zeros(max(g.n, 1), bool)
    flags[np.asarray(cover, np.int64)] = True
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return bool(np.all(flags[src] | flags[g.col]))


def prepare_pvc_batch(vc, stream, count=4096, budget=200_000, seed=11, rank=0, world=1):
    """The batched PVC workload: 4,096 graphs, n ~ U[40, 1500] (half G(n,p)
    with mean degree U[3, 8], half Chung-Lu 2.5), each queried at k = opt
    (yes) and k = opt - 1 (no).  opt comes from a first batched MVC launch
    under the same per-query node budget; graphs over budget there are
    dropped and counted.  Launch options are autotuned on the queries."""
    mix = gg.batch_pvc_mix(count, seed)
    if world > 1:   # this rank's share of the graphs, balanced by size
        mix = [mix[i] for i in shard_by_cost([g.n + g.m for g in mix], world)[rank]]
    dms = [vc.Graph.from_csr(h.row_ptr, h.col, stream=stream) for h in mix]
    t0 = time.perf_counter()
    sizes, _, status, _, mst = vc.solve_batch(dms, node_budget=budget, want_covers=False, raise_on_error=False)
    mvc_s = time.perf_counter() - t0
    solved = [i for i in range(len(mix)) if status[i] == 0]
    qg = [dms[i] for i in solved] * 2
    ks = [int(sizes[i]) for i in solved] + [int(sizes[i]) - 1 for i in solved]
    tuned, _, _ = vc.autotune(qg, ks, repeats=1, node_budget=budget)
    return {"mix": mix, "dms": dms, "sizes": sizes, "status": status, "solved": solved, "qg": qg, "ks": ks,
            "tuned": tuned, "mvc_s": mvc_s, "mvc_stats": mst, "budget": budget, "count": len(mix), "seed": seed,
            "total": count}


def search_block(vc, torch, prep, steps, hbm_peak, hbm_kind, l2_peak, flush, world=1, group=None):
    """The persistent search measured on the batched PVC workload at full
    size: `steps` launches of all its queries (each launch one root phase and
    one persistent search), L2 flushed before each.  The search kernel's time
    is its CUDA-event duration on the launching stream (recorded by the
    library around the launch); nodes/s and algorithmic bytes per node come
    from the kernel's own counters; the achieved rate is held against the
    measured HBM copy peak and the L2 read peak measured in this run."""
    qg, ks, tuned, budget = prep["qg"], prep["ks"], prep["tuned"], prep["budget"]
    ns = len(prep["solved"])
    for _ in range(2):   # the second call captures the search phase into a CUDA graph
        vc.solve_batch(qg, ks, opts=tuned, want_covers=False, raise_on_error=False)
    ms, wall, nodes, nbytes, wrong, over, launches = [], [], 0, 0, 0, 0, 0
    for _ in range(steps):
        flush.fill_(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, pyes, pst, _, bst = vc.solve_batch(qg, ks, opts=tuned, want_covers=False, raise_on_error=False)
        wall.append(time.perf_counter() - t0)
        ok = pst == 0
        wrong += int(np.sum(ok[:ns] & ~pyes[:ns])) + int(np.sum(ok[ns:] & pyes[ns:]))
        over += int((pst == vc.VC_EBUDGET).sum())
        ms.append(bst["ms_search"])
        nodes += bst["nodes"]
        nbytes += bst["search_bytes"]
        launches += bst["launches"]
    # ranks solve disjoint shards: the job's time is the slowest rank's
    c = combine_search({"queries": len(qg), "nodes": nodes, "ms_wall": sum(wall) * 1e3, "ms_kernel": sum(ms),
                        "wrong": wrong, "over": over, "bytes": nbytes, "dropped": prep["count"] - ns}, world, group)
    nodes, nbytes, wrong, over = c["nodes"], c["bytes"], c["wrong"], c["over"]
    ksec = c["ms_kernel"] / 1e3
    achieved = nbytes / ksec / 1e9
    out = {"workload": "pvc_batch_4096", "graphs": prep["total"], "seed": prep["seed"],
           "node_budget_per_query": budget, "dropped_over_budget_in_mvc_rank0": prep["count"] - ns,
           "queries": c["queries"], "steps": steps, "l2": "256 MiB write before every step",
           "kernel": "search_kernel", "ms_search_kernel": round(c["ms_kernel"] / steps, 3),
           "nodes_per_launch": nodes // steps, "nodes_per_s": round(nodes / ksec, 1),
           "queries_per_s": round(c["queries"] * steps / (c["ms_wall"] / 1e3), 1),
           "time_to_solution_ms": round(c["ms_wall"] / steps, 3),
           "over_budget_per_launch": over // steps, "wrong_answers": wrong,
           "bytes_per_node": round(nbytes / max(1, nodes), 1), "achieved_gbs": round(achieved, 3),
           "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": hbm_kind, "frac_hbm": round(achieved / hbm_peak, 6),
           "l2_peak_gbs": round(l2_peak, 1), "l2_peak_kind": "measured in this run (vc_measure_l2_read, 32 MiB)",
           "frac_l2": round(achieved / l2_peak, 6) if l2_peak > 0 else None,
           "traffic": kernel_traffic("search_kernel", "pvc_batch_4096"),
           "options": {f: getattr(tuned, f) for f in vc.TUNED_FIELDS}, "gpu_launches": launches}
    if world > 1:
        out.update(sharding=f"LPT over {world} ranks by n + m, host gather (gloo)",
                   per_rank_queries=c["per_rank_queries"])
    return out


def extra_pvc_batch(vc, stream, prep):
    """Batched against plain on the batched PVC workload: one launch for all
    queries against one launch per query (a 512-query sample), and the
    oracle over every host core on the same sample."""
    mix, dms, qg, ks, tuned, budget = prep["mix"], prep["dms"], prep["qg"], prep["ks"], prep["tuned"], prep["budget"]
    solved = prep["solved"]
    count = prep["count"]
    vc.solve_batch(qg[:64], ks[:64], opts=tuned, raise_on_error=False)
    t0 = time.perf_counter()
    psz, pyes, pst, covers, bst = vc.solve_batch(qg, ks, opts=tuned, raise_on_error=False)
    batch_s = time.perf_counter() - t0
    ns = len(solved)
    ok = pst == 0
    wrong = int(np.sum(ok[:ns] & ~pyes[:ns])) + int(np.sum(ok[ns:] & pyes[ns:]))
    bad_cover = sum(1 for j in range(ns) if ok[j] and not cover_ok(mix[solved[j]], covers[j]))
    # plain: one launch per query on a sample of the same queries
    rng = np.random.default_rng(3)
    sample = rng.choice(len(qg), size=min(512, len(qg)), replace=False)
    t0 = time.perf_counter()
    plain_ok = 0
    plain_err = {}   # status -> count (VC_EBUDGET: the search order differs between launches)
    for j in sample:
        try:
            y, _, _ = vc.solve_k(qg[j], ks[j], node_budget=budget, want_cover=True)
            plain_ok += int(y == (int(j) < ns))
        except vc.VcError as e:
            plain_err[str(e.status)] = plain_err.get(str(e.status), 0) + 1
    plain_s = time.perf_counter() - t0
    # the oracle on the same sample, over every host core
    cpu_all = cpu_oracle_all_cores([(mix[solved[int(j) % ns]], ks[int(j)]) for j in sample], budget=budget)
    return {"graphs": count, "node_budget_per_query": budget, "mvc_launch_s": round(prep["mvc_s"], 3),
            "dropped_over_budget_in_mvc": count - ns, "queries": len(qg),
            "batched_queries_per_s": round(int(ok.sum()) / batch_s, 1), "batched_s": round(batch_s, 3),
            "batched_over_budget": int((pst == vc.VC_EBUDGET).sum()), "wrong_answers": wrong,
            "covers_failing_edge_check": bad_cover, "batched_nodes_per_s": round(bst["nodes"] / batch_s, 1),
            "batched_options": {f: getattr(tuned, f) for f in vc.TUNED_FIELDS},
            "plain_sample": len(sample), "plain_queries_per_s": round(len(sample) / plain_s, 1),
            "plain_matching_answers": plain_ok, "plain_errors": plain_err, "cpu_oracle_all_cores": cpu_all}


def extra_c4_budget_study(vc, stream, prep, big=2_000_000, sample=32, max_s=120.0):
    """The batched PVC workload's graphs that exceeded the 200k-node budget
    in the minimum-cover pass, solved again in one batch under a 2M-node
    budget: how many finish, and, for a sample of those, the oracle's answer
    on every host core under the same budget (its rate is the CPU baseline;
    both must agree)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    dropped = [i for i in range(prep["count"]) if prep["status"][i] == vc.VC_EBUDGET]
    graphs = [prep["mix"][i] for i in dropped]
    dgs = [prep["dms"][i] for i in dropped]
    t0 = time.perf_counter()
    sizes, _, status, _, st = vc.solve_batch(dgs, node_budget=big, want_covers=False, raise_on_error=False)
    dev_s = time.perf_counter() - t0
    fin = [j for j in range(len(dropped)) if status[j] == 0]
    rng = np.random.default_rng(17)
    pick = sorted(rng.choice(len(fin), size=min(sample, len(fin)), replace=False).tolist()) if fin else []

    def one(j):
        g = graphs[fin[j]]
        try:
            return oracle.mvc(g.n, g.row_ptr, g.col, node_budget=big)[0]
        except oracle.OracleBudgetExceeded:
            return None

    agree = disagree = over = 0
    t1 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for j, want in zip(pick, ex.map(one, pick)):
            if want is None:
                over += 1
            elif want == int(sizes[fin[j]]):
                agree += 1
            else:
                disagree += 1
            if time.perf_counter() - t1 > max_s:
                break
    return {"graphs": prep["count"], "dropped_at_200k": len(dropped), "node_budget": big,
            "finished_at_2m": len(fin), "still_over": int(np.sum(status == vc.VC_EBUDGET)),
            "device_s": round(dev_s, 3), "device_nodes": st["nodes"],
            "oracle_sample": len(pick), "oracle_agree": agree, "oracle_disagree": disagree,
            "oracle_over_budget": over, "oracle_s": round(time.perf_counter() - t1, 3),
            "oracle_cores": os.cpu_count() or 1}


def induced_piece(g, lo: int, hi: int):
    """The subgraph induced by vertices [lo, hi), relabelled from 0."""
    u, v = gg.edges_of(g)
    keep = (u >= lo) & (u < hi) & (v >= lo) & (v < hi)
    return gg.from_edges(hi - lo, u[keep] - lo, v[keep] - lo)


def extra_component_heavy_full(vc, stream, peak, budget=100_000_000, copies=256, copy_n=48, chain=32):
    """The component-heavy shape at full size (256 copies of G(48, 0.12) on a
    32-vertex chain, about 12.3k vertices) under a node budget: it does not
    finish within it, so this measures the search rate and its roofline, and
    certifies what it can: the best cover the search had found when it
    stopped (an upper bound), beside a lower bound from disjoint induced
    subgraphs -- each copy and the chain, solved exactly (a cover of the
    whole graph covers each piece's edges, so the pieces' optima add up to a
    lower bound on the whole)."""
    g = gg.component_heavy(0, copies=copies, copy_n=copy_n, p=0.12, chain=chain)
    d = vc.Graph.from_csr(g.row_ptr, g.col, stream=stream)
    try:
        size, _, st = vc.solve_min(d, node_budget=budget)
        status = 0
    except vc.VcError as e:
        size, st, status = -1, e.stats, e.status
    d.close()
    ms = st["ms_search"]
    gbs = st["search_bytes"] / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    pieces = [induced_piece(g, 0, chain)]
    pieces += [induced_piece(g, chain + i * copy_n, chain + (i + 1) * copy_n) for i in range(copies)]
    dps = [vc.Graph.from_csr(h.row_ptr, h.col, stream=stream) for h in pieces]
    psz, _, pst, _, _ = vc.solve_batch(dps, want_covers=False, raise_on_error=False)
    for x in dps:
        x.close()
    lower = int(np.sum(psz)) if np.all(pst == 0) else None
    upper = size if status == 0 else st["best_found"]
    return {"n": g.n, "n_induced": st["n_induced"], "status": status, "answer": size, "node_budget": budget,
            "nodes": st["nodes"], "ms_search_kernel": round(ms, 3),
            "nodes_per_s": round(st["nodes"] / (ms / 1e3), 1) if ms > 0 else None,
            "component_branches": st["component_branches"], "workers": st["workers"], "team": st["team"],
            "certificate": {"upper_best_cover_found": upper,
                            "lower_disjoint_pieces": lower,
                            "gap": (upper - lower) if lower is not None else None,
                            "pieces": "the 32-vertex chain and each of the 256 copies, solved exactly"},
            "search_roofline": {"bound": "hbm", "kernel": "search_kernel", "achieved": round(gbs, 3),
                                "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 6),
                                "bytes_per_node": round(st["search_bytes"] / max(1, st["nodes"]), 1),
                   "crown_forced": st["crown_forced"], "crown_removed": st["crown_removed"]}}


def extra_ablation(vc, stream, budget=200_000_000):
    """The paper's ablation (Tables 2-4, Figure 4) on synthetic graphs: each
    optimisation switched off in turn, under a node budget (a run over it is
    reported with status VC_EBUDGET and the nodes it visited), plus the
    execution-time breakdown of the full method."""
    cases = {"component_heavy_8x48": gg.component_heavy(1, copies=8, copy_n=48, p=0.12, chain=2),
             "gnm_40_90_x100": gg.disjoint_union([gg.gnm(40, 90, 500 + s) for s in range(100)])}
    variants = [("all_on", dict(breakdown=1)), ("components_off", dict(use_components=0)),
                ("root_reduction_off", dict(disable_root_rules=1)), ("bounds_off", dict(disable_bounds=1)),
                ("dynamic_component_bounds_off", dict(disable_dyn_bounds=1)),
                ("crown_on", dict(crown=1)),
                ("load_balance_off", dict(load_balance=0))]
    out = {}
    for name, g in cases.items():
        d = vc.Graph.from_csr(g.row_ptr, g.col, stream=stream)
        vc.solve_min(d)
        rows = {}
        for vname, kw in variants:
            t0 = time.perf_counter()
            try:
                size, _, st = vc.solve_min(d, node_budget=budget, want_cover=False, **kw)
                status = 0
            except vc.VcError as e:
                size, st, status = -1, e.stats, e.status
            wall = time.perf_counter() - t0
            row = {"status": status, "answer": size, "s": round(wall, 4), "nodes": st["nodes"],
                   "component_branches": st["component_branches"], "comp_hist": st["comp_hist"],
                   "vertices_in_degree_array": st["n_induced"], "dtype_bytes": st["dtype_bytes"],
                   "workers": st["workers"], "team": st["team"],
                   "bytes_per_node": round(st["search_bytes"] / max(1, st["nodes"]), 1),
                   "crown_forced": st["crown_forced"], "crown_removed": st["crown_removed"]}
            if kw.get("breakdown"):
                ph = st["phase_cycles"]
                tot = sum(ph.values())
                row["breakdown"] = {k: round(v / tot, 4) for k, v in ph.items()} if tot else None
            rows[vname] = row
        d.close()
        out[name] = {"n": g.n, "node_budget": budget, "runs": rows}
    return out


def _pct(xs, q):
    return round(float(np.percentile(xs, q)), 3) if len(xs) else None


def extra_served_stream(vc, stream, count=1000, rates=(250.0, 1000.0, 4000.0), budget=100_000, seed=5):
    """Served stream: Chung-Lu requests (n log-uniform on [30, 20000],
    exponent U[2.2, 3.0], mean degree U[4, 10], maximum degree n / 4) with
    Poisson arrivals, at each offered rate.  Served: requests are submitted
    at their arrival times and the server is stepped continuously (real
    time).  Plain: one vc_load_csr + vc_solve_min + vc_free per request, FIFO;
    each request's service time is measured and its latency follows from the
    single-server queue (finish = max(arrival, previous finish) + service).
    Latency = retirement - arrival.  Both forms take the same requests under
    the same per-request node budget, and the server's size classes take
    every induced graph of the stream (no capacity refusal), so graphs/s is
    over an identical request set; latency percentiles are also given over
    the requests both forms answered."""
    tg = time.perf_counter()
    t_unit, specs = gg.stream_requests(count, seed, 1.0)
    graphs = [gg.chung_lu(n, gam, d, max(4.0, n / 4.0), s) for (n, gam, d, s) in specs]
    _log(f"served_stream: {count} graphs generated in {time.perf_counter() - tg:.1f} s")
    srv = vc.Server(stream=stream, node_budget=budget)
    for g in graphs[:32]:                       # warm-up
        srv.submit(g.row_ptr, g.col)
    srv.drain()
    out = {"requests": count, "node_budget_per_request": budget, "rates": []}
    served_ans = None
    served_lat = []
    for rate in rates:
        arr = np.asarray(t_unit) / rate
        lat = np.zeros(count)
        ans = {}
        t0 = time.perf_counter()
        i = 0
        while len(ans) < count:
            now = time.perf_counter() - t0
            while i < count and arr[i] <= now:
                srv.submit(graphs[i].row_ptr, graphs[i].col, tag=i)
                i += 1
            q, f, _ = srv.counts()
            if q or f:
                srv.step()
            elif i < count:
                time.sleep(max(0.0, min(arr[i] - now, 0.002)))
            for r in srv.poll():
                j = r["tag"]
                lat[j] = (time.perf_counter() - t0) - arr[j]
                ans[j] = (r["status"], r["size"], r["n_induced"])
        wall = time.perf_counter() - t0
        _log(f"served_stream: rate {rate}/s served in {wall:.2f} s")
        served_ans = ans
        served_lat.append(lat.copy())
        okm = np.array([ans[j][0] == 0 for j in range(count)])
        out["rates"].append({"offered_per_s": rate, "served_graphs_per_s": round(count / wall, 1),
                             "served_wall_s": round(wall, 3), "ok": int(okm.sum()),
                             "over_budget": int(sum(ans[j][0] == vc.VC_EBUDGET for j in range(count))),
                             "over_capacity": int(sum(ans[j][0] == vc.VC_ECAPACITY for j in range(count))),
                             "p50_ms": _pct(lat * 1e3, 50), "p95_ms": _pct(lat * 1e3, 95),
                             "p99_ms": _pct(lat * 1e3, 99)})
    sst = srv.stats()
    srv.close()
    # plain per-graph launches: service times
    service = np.zeros(count)
    plain_ans = {}
    for j, g in enumerate(graphs):
        t0 = time.perf_counter()
        d = vc.Graph.from_csr(g.row_ptr, g.col, stream=stream)
        try:
            size, _, _ = vc.solve_min(d, node_budget=budget)
            plain_ans[j] = (0, size)
        except vc.VcError as e:
            plain_ans[j] = (e.status, -1)
        d.close()
        service[j] = time.perf_counter() - t0
    _log(f"served_stream: plain service total {service.sum():.2f} s")
    for k, rate in enumerate(rates):
        arr = np.asarray(t_unit) / rate
        fin = np.zeros(count)
        prev = 0.0
        for j in range(count):
            prev = max(arr[j], prev) + service[j]
            fin[j] = prev
        lat = fin - arr
        out["rates"][k].update({"plain_graphs_per_s": round(count / (fin[-1] - arr[0]), 1),
                                "plain_p50_ms": _pct(lat * 1e3, 50), "plain_p95_ms": _pct(lat * 1e3, 95),
                                "plain_p99_ms": _pct(lat * 1e3, 99)})
    both = [j for j in range(count) if served_ans[j][0] == 0 and plain_ans[j][0] == 0]
    for k, rate in enumerate(rates):
        arr = np.asarray(t_unit) / rate
        fin = np.zeros(count)
        prev = 0.0
        for j in range(count):
            prev = max(arr[j], prev) + service[j]
            fin[j] = prev
        pl = (fin - arr)[both] * 1e3
        sl = served_lat[k][both] * 1e3
        out["rates"][k].update({"answered_by_both": len(both),
                                "served_p50_ms_both": _pct(sl, 50), "served_p99_ms_both": _pct(sl, 99),
                                "plain_p50_ms_both": _pct(pl, 50), "plain_p99_ms_both": _pct(pl, 99)})
    out["same_requests_same_budget"] = True
    out["answers_compared"] = len(both)
    out["answers_differing"] = sum(served_ans[j][1] != plain_ans[j][1] for j in both)
    out["plain_service_s"] = round(float(service.sum()), 3)
    out["server"] = {k: sst[k] for k in ("workers", "team", "dtype_bytes", "max_induced", "slices", "steps",
                                         "nodes", "ms_search", "ms_admit", "ms_retire", "resets")}
    return out


def ours_main(args, rank, world, local_rank):
    import torch
    import paper_2512_18334_gb300 as vc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)

    g = make_graph(rank)
    dg = vc.Graph.from_csr(g.row_ptr, g.col, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- warm-up (also checks the answer against the library's own verify path)
    for _ in range(max(args.warmup, 3)):
        size, cover, st = vc.solve_min(dg, **solve_options())
    flags = np.zeros(g.n, np.uint8)
    flags[cover] = 1
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert len(cover) == size and np.all(flags[src] | flags[g.col]), "cover check failed"

    # ---- timed: device-resident input, L2 flushed before each step
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, root_ms, search_ms, nodes, launches, search_bytes = [], [], [], 0, 0, 0
    for _ in range(args.steps):
        flush.fill_(0)
        ev0.record(stream)
        size_k, _, st = vc.solve_min(dg, want_cover=True, **solve_options())
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        root_ms.append(st["ms_root"])
        search_ms.append(st["ms_search"])
        nodes += st["nodes"]
        search_bytes += st["search_bytes"]
        launches += st["launches"]       # the L2-flush fill is torch's kernel, not counted
    barrier()
    clk = clocks.stop()
    total_ms, value = combine_over_ranks(sum(step_ms), args.steps, world)
    p99 = float(np.percentile(step_ms, 99))

    # ---- e2e: pinned host CSR -> vc_load_csr -> solve -> cover to host -> free
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    h2d = (rp_h.numel() + col_h.numel()) * 4
    e2e_ms, d2h = [], 0
    barrier()
    for _ in range(args.steps):
        flush.fill_(0)
        ev0.record(stream)
        h = vc.Graph.from_csr(rp_h.numpy(), col_h.numpy(), stream=stream)
        s2, cov2, _ = vc.solve_min(h, **solve_options())
        h.close()
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1))
        d2h = 4 * len(cov2) + 4
    barrier()
    e2e_total, e2e_value = combine_over_ranks(sum(e2e_ms), args.steps, world)

    # ---- roofline of the dominant kernel, timed by the library with CUDA
    # events on the launching stream
    peak, peak_kind = load_peaks()
    mean_root_ms = statistics.mean(root_ms)
    mean_search_ms = statistics.mean(search_ms)
    if mean_search_ms > mean_root_ms:
        kname = "search_kernel"
        algo = search_bytes / args.steps
        achieved = algo / (mean_search_ms / 1e3) / 1e9
        ms_launch = mean_search_ms
    else:
        kname = "root_cluster_kernel" if g.n >= 8192 else "root_kernel"
        algo = root_algorithmic_bytes(g, st)
        achieved = algo / (mean_root_ms / 1e3) / 1e9
        ms_launch = mean_root_ms
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 3),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 6), "traffic": kernel_traffic(kname),
                "algorithmic_bytes": int(algo), "ms_per_launch": round(ms_launch, 4)}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and WORKLOAD["workload"] == "chung_lu_50k":
        v, ms, osize = cpu_oracle_run(steps=2, warmup=0)
        assert osize == size, (osize, size)
        cpu = {"value": round(v, 6), "unit": "graphs/s", "cores": 1, "kind": "oracle",
               "sample": "2 solves of the same workload graph, single thread", "host": host_cpu()}

    # ---- the persistent search on the batched PVC workload (every rank
    # solves its shard of the 4,096 graphs)
    search, prep = None, None
    if not args.no_search:
        l2_peak = vc.measure_l2_read(32 << 20, 50, 5, stream=stream)
        group = host_group() if world > 1 else None
        prep = prepare_pvc_batch(vc, stream, rank=rank, world=world)
        search = search_block(vc, torch, prep, args.search_steps, peak, peak_kind, l2_peak, flush, world, group)
        if rank == 0:
            _log(f"search: {json.dumps(search, default=_json_default)}")

    if rank == 0 and args.c4_study and prep is not None and world == 1:
        study = extra_c4_budget_study(vc, stream, prep)
        _log(f"c4_study: {json.dumps(study, default=_json_default)}")
        if search is not None:
            search["budget_study"] = study

    also = None
    if rank == 0 and not args.no_extra:
        legs = [("small_graphs", lambda: extra_workloads(vc, torch, stream, peak)),
                ("served_stream", lambda: extra_served_stream(vc, stream, count=args.stream_requests)),
                ("pvc_batch_4096", lambda: extra_pvc_batch(vc, stream, prep if prep and world == 1
                                                           else prepare_pvc_batch(vc, stream))),
                ("component_heavy_256x48", lambda: extra_component_heavy_full(vc, stream, peak)),
                ("ablation", lambda: extra_ablation(vc, stream))]
        also = {}
        for name, fn in legs:
            t0 = time.perf_counter()
            try:
                r = fn()
            except Exception as e:   # a context leg never takes the headline line down with it
                r = {"error": f"{type(e).__name__}: {e}"}
            r["wall_s"] = round(time.perf_counter() - t0, 2)
            if name == "small_graphs":
                also.update(r)
            else:
                also[name] = r
            print(f"[bench] {name}: {json.dumps(r, default=_json_default)}", file=sys.stderr, flush=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "graphs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "impl": "ours",
            "config": dict(WORKLOAD, seed=(1000 if WORKLOAD["workload"] == "chung_lu_50k" else 1) + rank,
                           answer=size, n_induced=st["n_induced"],
                           forced=st["forced"], l2="256 MiB write before every timed step",
                           parallelism=f"replicas x{world}"),
            "p99_ms": round(p99, 4),
            "nodes_per_sec": round(nodes / (total_ms / 1e3), 1),
            "ms_root_kernel": round(mean_root_ms, 4),
            "ms_search_kernel": round(statistics.mean(search_ms), 4),
            "root_rounds": st["root_rounds"], "root_cycles": st["root_cycles"],
            "e2e": {"value": round(e2e_value, 3), "unit": "graphs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "search": search,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": launches,
            "also": also,
        }
        print(json.dumps(line, default=_json_default), flush=True)
    dg.close()
    if prep is not None:
        for d in prep["dms"]:
            d.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the context workloads")
    ap.add_argument("--no-search", action="store_true", help="skip the search block (batched PVC workload)")
    ap.add_argument("--search-steps", type=int, default=3, help="timed launches of the search block")
    ap.add_argument("--c4-study", action="store_true",
                    help="also solve the batched workload's over-budget graphs under a 2M-node budget")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="chung_lu_50k")
    ap.add_argument("--stream-requests", type=int, default=1000,
                    help="requests in the served-stream context measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    rank, world, local_rank = dist_env()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the ranks under torchrun (same arguments)
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    if world != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but {world} ranks were started")
    if args.impl == "reference":
        reference_main(args, rank, world)
    else:
        ours_main(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
