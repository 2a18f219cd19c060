#!/usr/bin/env python
"""Benchmark of the D-RSF batch update on one GB300.

Workload (default): R-MAT scale 22, edge factor 16, Graph500 initiator
(0.57, 0.19, 0.19, 0.05), ids permuted, seed 5 (4,194,304 vertices, ~64M
undirected edges, synthetic stand-in for the paper's Kronecker graphs); the
initial forest is the FIFO-BFS forest from each component's smallest id.
One step = one 100K-edge insert batch (uniform new pairs) followed by one
100K-edge delete batch (50% tree edges of the current forest, 50% non-tree
edges), applied through the C ABI.  Metric: updates/s = applied updates per
second over exactly K timed steps (CUDA events, L2 flushed between steps).

The batches follow one trajectory: an untimed planning pass on the GPU
generates each batch from the current graph and forest, then a fresh handle
replays the same batches for timing (the update is deterministic, so the
timed run sees the same states; the final parent arrays are compared).

Prints one JSON line (rank 0).  --impl reference times the serial CPU oracle
on the same workload instead.  With --gpus N > 1 (torchrun) every rank runs
an independent replica (the update of one graph does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "updates/s (insert + delete, R-MAT scale 22, 100K-update batches)"
UNIT = "updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="rmat22",
                   choices=["rmat22", "rmat20", "grid4096", "er-small", "batched256", "serving"])
    p.add_argument("--requests", type=int, default=400, help="serving: requests in the trace")
    p.add_argument("--load", type=float, default=0.9, help="serving: arrival rate / synchronous capacity")
    p.add_argument("--loads", default="0.5,0.7,0.9", help="serving: the load points of the latency curve")
    p.add_argument("--batch", type=int, default=0, help="batch size (default per workload)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--euler", action="store_true", help="Euler-tour path marks (Algorithm 3)")
    p.add_argument("--sweep", default="", help="comma-separated batch sizes: one JSON line per size")
    p.add_argument("--no-variants", action="store_true", help="skip the SG / HS replacement-variant timing")
    return p.parse_args()


# ------------------------------------------------------------ workloads

_GRAPHS = {}


def make_graph(name):
    """The workload's graph and trajectory parameters (generated once per
    process)."""
    if name not in _GRAPHS:
        _GRAPHS[name] = _make_graph(name)
    return _GRAPHS[name]


def _make_graph(name):
    import workloads
    if name == "rmat22":
        return workloads.rmat_graph(22, 16, seed=5), dict(tree_frac=0.5, local=0, batch=100_000)
    if name == "rmat20":
        return workloads.rmat_graph(20, 16, seed=2), dict(tree_frac=0.5, local=0, batch=100_000)
    if name == "grid4096":
        return workloads.grid_graph(4096, 4096, seed=3), dict(tree_frac=0.9, local=64, batch=100_000)
    return workloads.er_graph(20_000, 25_000, seed=1), dict(tree_frac=0.5, local=0, batch=2000)


def workload_config(name, g, b):
    desc = {
        "rmat22": "R-MAT scale 22, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), ids permuted, seed 5",
        "rmat20": "R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), ids permuted, seed 2",
        "grid4096": "4096x4096 grid, p=0.6, 0.1% shortcuts, seed 3; deletes 90% tree, inserts within 64 cells",
        "er-small": "Erdos-Renyi n=20,000 m=25,000 seed 1",
    }[name]
    return {"workload": desc, "vertices": int(g.n), "edges": int(g.m), "batch": int(b),
            "step": f"one {b}-edge insert batch + one {b}-edge delete batch",
            "initial_forest": "FIFO BFS from each component's smallest id",
            "reversal": ("euler-tour intervals" if getattr(ARGS, "euler", False)
                         else "walks up to 64 edges, pointer-doubling marks beyond"),
            "root_search": os.environ.get("DRSF_JUMP", "asynchronous pointer doubling"),
            "l2": "flushed between timed steps (256 MB write)"}


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        load = [r for r in rows if r[2] > 0.3 * max(x[2] for x in rows)] or rows
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ distributed

def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(units: float, seconds: float):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([units, seconds], dtype=torch.float64, device=dev)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


# ------------------------------------------------------------ algorithmic bytes

def phase_bytes(st: dict, n: int, op: int) -> dict:
    """Algorithmic bytes per phase of one batch, from the batch's counters:
    each data item the method must touch, counted once per pass, uncached
    (per-unit figures: a0 24 per batch edge, a1 insert 16 + two 32-byte index
    probes per applied edge, a1 delete two probes + an 8-byte tombstone, a2 4
    per batch edge for the cut and 12 per doubling step taken (at most 12 per
    affected vertex and doubling round),
    a3 12 per scanned row + 8 per scanned entry + 8 per candidate and 24 per
    candidate and hooking round, a4 64 r log2 r, a5 13 per active vertex and
    marking round + 12 per reversed vertex, a6 8 per vertex of the pass)."""
    b, a = st["batch_len"], st["applied"]
    out = {"begin": 8 * b}
    if op == 0:
        out["ins_claim"] = 16 * b + 64 * a
        out["ins_place"] = 16 * a + 8 * st["candidates"]
        out["active"] = 8 * n
    else:
        aff = st["affected"]
        out["del_claim"] = 16 * b + 72 * a + 4 * b
        out["affected"] = 8 * n
        # each doubling step taken (a visit: read J, gather J[J], write) counts
        # 12 bytes; the steps taken stay below affected x doubling rounds
        out["jump"] = 12 * st.get("jump_visits", aff * max(st["jump_rounds"], 1))
        if st.get("detach_levels", 0) > 0:
            # top-down search instead of pointer jumping: per scanned entry
            # the column and the parent gather, per detached vertex its
            # representative, list slot and row record
            out["jump"] = 8 * st["detach_entries"] + 24 * aff
            out["affected"] = 0
        out["scan"] = 12 * st["detached"] + 8 * st["scanned"] + 8 * st["candidates"]
        out["active"] = 8 * aff
    c, ner = st["candidates"], st["replacement"]
    out["hook"] = 24 * c * max(st["hook_rounds"], 1)
    out["orient"] = int(64 * ner * max(math.log2(max(ner, 2)), 1))
    out["mark"] = 13 * st["active"] * st["mark_rounds"]
    out["reverse"] = 12 * st["reversed"] + 8 * ner
    return out


def ncu_traffic(kernel_phase: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken
    on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel_phase)
        if not d:
            return None
        src = os.path.join(ROOT, d["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return d["bytes_per_launch"] if sha == d["source_sha"] else None
    except Exception:
        return None


# ------------------------------------------------------------ our arm

def plan(g, cfg, steps, b, seed):
    """Untimed pass on the GPU that generates the trajectory's batches."""
    import torch
    import paper_2607_20211_gb300 as drsf
    import workloads
    f = drsf.DynamicForest(g.n, torch.from_numpy(g.edges()).cuda(), torch.from_numpy(g.parent).cuda())
    tr = workloads.Trajectory(g, seed, tree_frac=cfg["tree_frac"], local=cfg["local"])
    out = []
    first = []   # parent arrays after the first step's two batches
    for k in range(steps):
        pair = []
        for op in (0, 1):
            batch = tr.next_batch(op, b)
            f.apply(op, torch.from_numpy(batch).cuda())
            st = f.stats()
            par = f.parent().cpu().numpy()
            tr.advance(batch, op, par)
            pair.append((batch, st))
            if k == 0:
                first.append(par.copy())
        out.append(pair)
    final = f.parent().cpu().numpy()
    f.close()
    return out, final, first


def run_ours(args, rank, ws, local):
    import torch
    import paper_2607_20211_gb300 as drsf
    torch.cuda.set_device(local)
    drsf.build()
    g, cfg = make_graph(args.workload)
    b = args.batch or cfg["batch"]
    K, W = args.steps, args.warmup
    steps, final_plan, first_parents = plan(g, cfg, W + K, b, seed=5)
    dev_batches = [[torch.from_numpy(p[0]).cuda() for p in s] for s in steps]
    edges_d = torch.from_numpy(g.edges()).cuda()
    parent_d = torch.from_numpy(g.parent).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    flags = drsf.DETERMINISTIC | (drsf.EULER_REVERSAL if args.euler else 0)
    f = drsf.DynamicForest(g.n, edges_d, parent_d, flags=flags)
    for s in range(W):
        for op in (0, 1):
            f.apply(op, dev_batches[s][op])
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        f.apply(0, dev_batches[W + k][0])
        ev[k][1].record(stream)
        f.apply(1, dev_batches[W + k][1])
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    barrier()
    final = f.parent().cpu().numpy()
    f.close()
    # per-phase device times: the same W + K steps replayed on a fresh
    # handle with every phase bracketed by CUDA events (direct launches:
    # events cannot sit between the kernels of a captured graph)
    f = drsf.DynamicForest(g.n, edges_d, parent_d, flags=flags)
    for s in range(W):
        for op in (0, 1):
            f.apply(op, dev_batches[s][op])
    torch.cuda.synchronize()
    f.profile_start(2 * K + 4)
    for k in range(K):
        flush.zero_()
        f.apply(0, dev_batches[W + k][0])
        f.apply(1, dev_batches[W + k][1])
    torch.cuda.synchronize()
    prof = f.profile_stop()
    if not np.array_equal(f.parent().cpu().numpy(), final_plan):
        raise RuntimeError("profiled replay diverged from the planning pass")
    # static rebuild of the final graph from scratch (the plain alternative)
    st_ms = []
    levels = 0
    for rep_i in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, levels = f.static_forest(with_levels=True) if rep_i == 0 else (*f.static_forest(), levels)
        e1.record(stream)
        torch.cuda.synchronize()
        st_ms.append(e0.elapsed_time(e1))
    f.close()
    if not np.array_equal(final, final_plan):
        raise RuntimeError("timed replay diverged from the planning pass")
    variants = None if args.no_variants else replacement_variants(g, edges_d, parent_d, dev_batches, W, min(K, 5),
                                                                   flush, stream)
    ins_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    del_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    step_ms = [i + d for i, d in zip(ins_ms, del_ms)]
    applied_i = sum(steps[W + k][0][1]["applied"] for k in range(K))
    applied_d = sum(steps[W + k][1][1]["applied"] for k in range(K))
    total_s = sum(step_ms) / 1e3
    units, secs = aggregate(float(applied_i + applied_d), total_s)

    # roofline of the dominant phase (kernel), from live events + the
    # algorithmic byte model over the same K steps
    pbytes = {}
    opbytes = {"insert": {}, "delete": {}}
    for k in range(K):
        for op, oname in ((0, "insert"), (1, "delete")):
            for ph, by in phase_bytes(steps[W + k][op][1], g.n, op).items():
                pbytes[ph] = pbytes.get(ph, 0) + by
                opbytes[oname][ph] = opbytes[oname].get(ph, 0) + by
    phases = {}
    for oname in ("insert", "delete"):
        for ph, (ms, nl) in prof[oname].items():
            t = phases.get(ph, (0.0, 0))
            phases[ph] = (t[0] + ms, t[1] + nl)
    dom = max(phases, key=lambda p: phases[p][0])
    dom_ms, dom_launch = phases[dom]
    per_launch_bytes = pbytes.get(dom, 0) / max(dom_launch, 1)
    per_launch_ms = dom_ms / max(dom_launch, 1)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "phase_timing": "CUDA events around each phase over the same K steps, replayed on a fresh handle "
                                "with direct launches (the timed run replays captured CUDA graphs)",
                "frac": round(achieved / peak, 4), "traffic": ncu_traffic(dom),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": int(per_launch_bytes),
                "ms_per_launch": round(per_launch_ms, 5)}
    # whole step: every phase's algorithmic bytes over the timed step time
    step_bytes = sum(pbytes.values()) / K
    step_gbs = step_bytes / (secs / K) / 1e9 if secs > 0 else 0.0
    roofline["step"] = {"algorithmic_bytes": int(step_bytes), "achieved": round(step_gbs, 1),
                        "frac": round(step_gbs / peak, 4), "ms": round(secs / K * 1e3, 4)}
    step_total_ms = sum(v[0] for v in phases.values())
    phase_table = {}
    for oname in ("insert", "delete"):
        phase_table[oname] = {
            p: {"ms_per_batch": round(v[0] / K, 4), "share_of_step": round(v[0] / step_total_ms, 4),
                "launches": int(v[1]),
                "GBps": round(opbytes[oname].get(p, 0) / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 else None}
            for p, v in prof[oname].items() if v[1] > 0}
    def _mean(op, key):
        return round(float(np.mean([steps[W + k][op][1][key] for k in range(K)])), 1)
    batch_stats = {oname: {key: _mean(op, key) for key in (
        "applied", "tree_cut", "affected", "detached", "scanned", "candidates", "hook_rounds", "replacement",
        "rank_rounds", "active", "reversed", "mark_rounds", "jump_rounds", "jump_visits", "detach_levels",
        "detach_entries", "core_arcs")} for op, oname in ((0, "insert"),
                                                                                        (1, "delete"))}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        f = drsf.DynamicForest(g.n, edges_d, parent_d)
        host = [[np.ascontiguousarray(p[0]) for p in s] for s in steps]
        for s in range(W):
            for op in (0, 1):
                f.apply_host(op, host[s][op])
        f.stats()
        barrier()
        tt = 0.0
        h2d = 0
        for k in range(K):
            t0 = time.perf_counter()
            f.apply_host(0, host[W + k][0])
            f.apply_host(1, host[W + k][1])
            st = f.stats()   # device -> host read of the step's result counters
            tt += time.perf_counter() - t0
            h2d += host[W + k][0].nbytes + host[W + k][1].nbytes
        barrier()
        f.close()
        eu, es = aggregate(float(applied_i + applied_d), tt)
        e2e = {"value": round(eu / es, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d // K),
               "d2h_bytes_per_step": 152, "ms_per_step": round(tt / K * 1e3, 4),
               "path": "drsf_apply_host (pinned staging) + drsf_stats read-back"}
        # the same steps with the whole updated forest F' read back to the
        # host every step (drsf_parent into a device buffer, then one copy
        # to pinned host memory): the full host-visible cost of an update
        f = drsf.DynamicForest(g.n, edges_d, parent_d)
        pbuf = torch.empty(g.n, dtype=torch.int32, device="cuda")
        phost = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
        for s in range(W):
            for op in (0, 1):
                f.apply_host(op, host[s][op])
        f.stats()
        barrier()
        tp = 0.0
        for k in range(K):
            t0 = time.perf_counter()
            f.apply_host(0, host[W + k][0])
            f.apply_host(1, host[W + k][1])
            st = f.stats()
            phost.copy_(f.parent(pbuf), non_blocking=True)
            torch.cuda.current_stream().synchronize()
            tp += time.perf_counter() - t0
        barrier()
        if not np.array_equal(phost.numpy(), final_plan):
            raise RuntimeError("e2e replay with read-back diverged from the planning pass")
        f.close()
        pu, ps = aggregate(float(applied_i + applied_d), tp)
        e2e["with_parent_readback"] = {"value": round(pu / ps, 1), "unit": UNIT, "ms_per_step": round(tp / K * 1e3, 4),
                                       "d2h_bytes_per_step": 152 + 4 * g.n,
                                       "path": "the same + drsf_parent and a copy of F' to pinned host memory"}
    clocks = clk.stop()

    cpu = None
    parity0 = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, parity0 = cpu_baseline(g, steps, first_parents)
    if rank != 0:
        return
    lat = sorted(ins_ms + del_ms)
    line = {
        "metric": METRIC if args.workload == "rmat22" else f"updates/s ({args.workload}, {b}-update batches)",
        "value": round(units / secs, 1), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": round(secs / K * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {**workload_config(args.workload, g, b), "parallelism": "replicas" if ws > 1 else "single"},
        "insert_updates_per_s": round(applied_i / (sum(ins_ms) / 1e3), 1),
        "delete_updates_per_s": round(applied_d / (sum(del_ms) / 1e3), 1),
        "batch_latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                             "p99": round(float(np.percentile(lat, 99)), 4),
                             "insert_p50": round(float(np.median(ins_ms)), 4),
                             "delete_p50": round(float(np.median(del_ms)), 4)},
        "static_rebuild": {"ms": round(float(np.median(st_ms[1:])), 4), "bfs_levels": int(levels),
                           "what": "components by hook-and-compress + multi-source BFS from component minima, "
                                   "on the final graph, same GPU",
                           "x_insert_batch": round(float(np.median(st_ms[1:])) / float(np.median(ins_ms)), 2),
                           "x_delete_batch": round(float(np.median(st_ms[1:])) / float(np.median(del_ms)), 2)},
        "replacement_variants": variants,
        "roofline": roofline, "phases": phase_table, "batch_stats": batch_stats, "e2e": e2e,
        "cpu_baseline": cpu,
        "parity_step0": parity0,
        "gpu_launches": int(sum(v[1] for v in phases.values())),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def replacement_variants(g, edges_d, parent_d, dev_batches, W, K, flush, stream):
    """Insert and delete batch times with each replacement-edge variant
    forced (supergraph reduction vs hooking on every cross edge, Section
    III), replaying the same first W + K steps on fresh handles."""
    import torch
    import paper_2607_20211_gb300 as drsf
    out = {}
    for name, flag in (("sg", drsf.REPL_SG), ("hs", drsf.REPL_HS)):
        f = drsf.DynamicForest(g.n, edges_d, parent_d, flags=drsf.DETERMINISTIC | flag)
        ms = {0: [], 1: []}
        cands = {0: [], 1: []}
        for k in range(W + K):
            for op in (0, 1):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                f.apply(op, dev_batches[k][op])
                e1.record(stream)
                st = f.stats()
                if k >= W:
                    ms[op].append(e0.elapsed_time(e1))
                    cands[op].append(st["candidates"])
        f.close()
        out[name] = {"insert_ms": round(float(np.median(ms[0])), 4), "delete_ms": round(float(np.median(ms[1])), 4),
                     "insert_candidates": int(np.mean(cands[0])), "delete_candidates": int(np.mean(cands[1]))}
    out["what"] = (f"median batch time over {K} steps after {W} warm-up, each variant forced; the default "
                   "picks per batch (SG when the key edges exceed n/16)")
    return out


def run_batched(args, rank, ws, local):
    """256 independent graphs (n log-uniform in [1K, 256K], half Erdos-Renyi,
    half R-MAT, average degree uniform in [4, 16], seed 4); each step gives
    every graph an insert batch then a delete batch (together 1-10% of its
    m, 60/40, deletes 50% tree edges).  Batched form: one launch sequence
    over the disjoint union of the graphs (ids offset per graph); compared
    with one launch sequence per graph (256 handles) on the same GPU."""
    import torch
    import paper_2607_20211_gb300 as drsf
    import workloads
    torch.cuda.set_device(local)
    drsf.build()
    K, W = args.steps, args.warmup
    graphs = workloads.batched_graphs(256, seed=4)
    U = workloads.Union(graphs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    edges_u, par_u = dev(workloads.keys_to_edges(U.keys)), dev(U.parent)
    # planning pass on the union handle: per-graph batches from per-graph state
    f = drsf.DynamicForest(U.n, edges_u, par_u)
    trs = [workloads.Trajectory(g, seed=(4 << 20) + i) for i, g in enumerate(graphs)]
    plan_steps = []
    for s in range(W + K):
        budgets = workloads.batched_budgets(graphs, seed=4 + 7919 * s)
        pair = []
        for op in (0, 1):
            per = [tr.next_batch(op, b[op]) for tr, b in zip(trs, budgets)]
            f.apply(op, dev(np.concatenate([U.shift(i, b) for i, b in enumerate(per)])))
            parts = U.split(f.parent().cpu().numpy())
            for tr, b, p in zip(trs, per, parts):
                tr.advance(b, op, p)
            pair.append(per)
        plan_steps.append(pair)
    final_plan = f.parent().cpu().numpy()
    f.close()
    ubat = [[dev(np.concatenate([U.shift(i, b) for i, b in enumerate(pair[op])])) for op in (0, 1)]
            for pair in plan_steps]
    gbat = [[[dev(b) for b in pair[op]] for op in (0, 1)] for pair in plan_steps]
    updates = sum(sum(len(b) for b in pair[op]) for pair in plan_steps[W:] for op in (0, 1))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(apply_step):
        tot = 0.0
        for k in range(W + K):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            apply_step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= W:
                tot += e0.elapsed_time(e1)
        return tot / 1e3

    # every form sizes its per-batch buffers for the largest batch first, so
    # no timed step grows them (a growth synchronises, reallocates and drops
    # the captured launch sequences)
    umax = max(int(b.shape[0]) for pair in ubat for b in pair)
    f = drsf.DynamicForest(U.n, edges_u, par_u)
    f.reserve(umax)
    barrier()
    t_union = timed(lambda k: (f.apply(0, ubat[k][0]), f.apply(1, ubat[k][1])))
    final = f.parent().cpu().numpy()
    f.close()
    if not np.array_equal(final, final_plan):
        raise RuntimeError("batched replay diverged from the planning pass")

    # persistent per-graph kernels (drsf_apply_batched), schedule from the
    # autotuner (cached per size class and op)
    from paper_2607_20211_gb300 import autotune
    voff = U.offsets.astype(np.int64)
    boffs = [[np.concatenate([[0], np.cumsum([len(b) for b in pair[op]])]).astype(np.int64) for op in (0, 1)]
             for pair in plan_steps]
    sig = autotune.signature(voff)
    sched = autotune.load(sig)
    tuned_now = sched is None
    if sched is None:
        f = drsf.DynamicForest(U.n, edges_u, par_u)
        f.apply(0, ubat[0][0])
        e1 = f.export_edges().clone()
        p1 = f.parent().clone()
        f.close()
        sched = autotune.tune(U.n, {0: (edges_u, par_u), 1: (e1, p1)}, voff,
                              {0: (ubat[0][0], boffs[0][0]), 1: (ubat[0][1], boffs[0][1])},
                              log=lambda m: print(m, file=sys.stderr))
        del e1, p1
    f = drsf.DynamicForest(U.n, edges_u, par_u)
    f.reserve(umax)
    t_persist = timed(lambda k: (f.apply_batched(0, ubat[k][0], voff, boffs[k][0], sched[0]),
                                 f.apply_batched(1, ubat[k][1], voff, boffs[k][1], sched[1])))
    final_p = f.parent().cpu().numpy()
    f.close()
    if not np.array_equal(final_p, final_plan):
        raise RuntimeError("persistent per-graph kernels diverged from the grid-wide path")
    hs = [drsf.DynamicForest(g.n, dev(g.edges()), dev(g.parent)) for g in graphs]
    for i, h in enumerate(hs):
        h.reserve(max(int(gbat[k][op][i].shape[0]) for k in range(W + K) for op in (0, 1)))

    def per_graph(k):
        for op in (0, 1):
            for h, b in zip(hs, gbat[k][op]):
                h.apply(op, b)
    t_each = timed(per_graph)
    parts = [h.parent().cpu().numpy() for h in hs]
    for h in hs:
        h.close()
    same = all(np.array_equal(a, b) for a, b in zip(parts, U.split(final)))
    if not same:
        raise RuntimeError("per-graph results differ from the batched form")
    u1, s1 = aggregate(float(updates), t_union)
    u2, s2 = aggregate(float(updates), t_each)
    u3, s3 = aggregate(float(updates), t_persist)
    if rank != 0:
        return
    line = {"metric": "updates/s (256 independent graphs, batched form)", "value": round(u3 / s3, 1),
            "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": round(s3 / K * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "256 graphs, n log-uniform [1K, 256K], half ER half R-MAT, degree U[4,16], "
                                   "seed 4; per step per graph: insert + delete batches of 1-10% of m (60/40)",
                       "vertices": U.n, "edges": int(len(U.keys)), "updates_per_step": updates // K,
                       "l2": "flushed between timed steps (256 MB write)"},
            "form": "persistent per-graph kernels (one thread-block cluster per graph, size-class queues, "
                    "captured CUDA graph)",
            "tuned_schedule": {("insert" if op == 0 else "delete"): [
                {"max_vertices": c[0], "block_threads": c[1], "blocks_per_sm": c[2], "cluster_blocks": c[3]}
                for c in sched[op]]
                for op in (0, 1)},
            "tuned_this_run": tuned_now,
            "union_grid_path": {"value": round(u1 / s1, 1), "ms_per_step": round(s1 / K * 1e3, 4),
                                "what": "the grid-wide launch sequence over the disjoint union"},
            "per_graph_launch_sequences": {"value": round(u2 / s2, 1), "ms_per_step": round(s2 / K * 1e3, 4),
                                           "handles": len(graphs)},
            "persistent_over_union": round((u3 / s3) / (u1 / s1), 3),
            "persistent_over_per_graph": round((u3 / s3) / (u2 / s2), 2),
            "batched_over_per_graph": round((u1 / s1) / (u2 / s2), 2),
            "results_identical": bool(same)}
    print(json.dumps(line), flush=True)


def run_serving(args, rank, ws, local):
    """Serving: a resident R-MAT scale-22 graph plus 64 tenant R-MAT graphs
    (scales 14-18, uniform), all kept on the device under a 120 GB budget; a
    Poisson stream of update batches (sizes log-uniform in [100, 1M], 60%
    insert / 40% delete, tenant Zipf(1.1) with rank 1 the resident graph,
    seed 5).  The continuous-batching server is compared with synchronous
    one-batch-at-a-time apply on the same trace and arrival times."""
    import math
    import torch
    import paper_2607_20211_gb300 as drsf
    import workloads
    from paper_2607_20211_gb300 import serve
    torch.cuda.set_device(local)
    drsf.build()
    rng = np.random.default_rng(5)
    graphs = {0: workloads.rmat_graph(22, 16, seed=5)}
    for i in range(1, 65):
        graphs[i] = workloads.rmat_graph(int(rng.integers(14, 19)), 16, seed=5000 + i)
    order = [0] + list(rng.permutation(np.arange(1, 65)))
    zipf = np.array([1.0 / (k + 1) ** 1.1 for k in range(65)])
    zipf /= zipf.sum()
    # the trace: batches drawn along each tenant's own trajectory (planning on the GPU)
    hs = {t: drsf.DynamicForest(g.n, torch.from_numpy(g.edges()).cuda(), torch.from_numpy(g.parent).cuda())
          for t, g in graphs.items()}
    trs = {t: workloads.Trajectory(g, seed=(5 << 20) + t) for t, g in graphs.items()}
    reqs = []
    for rid in range(args.requests):
        t = int(order[rng.choice(65, p=zipf)])
        op = int(rng.random() < 0.4)
        size = int(round(math.exp(rng.uniform(math.log(100), math.log(1_000_000)))))
        tr = trs[t]
        if op == 1:
            tr.parent = hs[t].parent().cpu().numpy()
        batch = tr.next_batch(op, size)
        hs[t].apply(op, torch.from_numpy(batch).cuda())
        tr.keys = workloads.apply_keys(tr.keys, batch, op)
        reqs.append(serve.Request(rid, t, op, batch, 0.0))
    for h in hs.values():
        h.close()
    tenants = {t: (g.n, g.edges(), g.parent) for t, g in graphs.items()}
    # capacity of the synchronous path (everything queued at time 0)
    done0, hs0 = serve.run_synchronous(tenants, reqs)
    for h in hs0.values():
        h.close()
    cap = len(reqs) / (max(d.t_done for d in done0))

    def new_server():
        srv = serve.Server(budget_bytes=120 << 30, slots=8, coalesce=True, reserve_edges=1_000_000)
        for t, (n, e, p) in tenants.items():
            srv.add_tenant(t, n, e, p)
        srv.admit_all()
        return srv

    def close_server(srv):
        srv.close()

    # warm-up of both forms (first launches, captures, allocator) on the
    # first quarter of the trace, not timed
    warm = reqs[: max(1, len(reqs) // 4)]
    _, hw = serve.run_synchronous(tenants, warm)
    for h in hw.values():
        h.close()
    srv_w = new_server()
    srv_w.run(warm)
    close_server(srv_w)
    # the latency curve: Poisson arrivals at each load (x synchronous
    # capacity), server and synchronous apply on the same trace
    loads = [float(x) for x in args.loads.split(",") if x] or [args.load]
    if args.load not in loads:
        loads.append(args.load)
    curve = {}
    same = None
    srv_main = sy_main = None
    for load in loads:
        lam = load * cap
        arr = np.cumsum(np.random.default_rng(5 + int(load * 100)).exponential(1.0 / lam, len(reqs)))
        timed = [serve.Request(r.rid, r.tenant, r.op, r.batch, float(a)) for r, a in zip(reqs, arr)]
        done_s, hs1 = serve.run_synchronous(tenants, timed)
        for h in hs1.values():
            h.close()
        srv = new_server()
        done_c = srv.run(timed)
        sv, sy = serve.summarize(done_c), serve.summarize(done_s)
        curve[str(load)] = {"arrival_rate_per_s": round(lam, 2), "server": sv, "synchronous": sy}
        if load == args.load:
            srv_main, sy_main = sv, sy
            # each tenant's result in the mix equals its applied log replayed alone
            same = True
            for t, g in graphs.items():
                _, par_mix = srv.state(t)
                f = drsf.DynamicForest(g.n, torch.from_numpy(g.edges()).cuda(), torch.from_numpy(g.parent).cuda())
                for op, b in srv.tenants[t].log:
                    f.apply_host(op, b)
                same &= bool(np.array_equal(f.parent().cpu().numpy(), par_mix))
                f.close()
            coalesced = int(sum(len(t.log) for t in srv.tenants.values()))
            evictions = srv.evictions
        close_server(srv)
    # saturation: everything queued at time 0 (capacity of each form)
    srv2 = new_server()
    done_c0 = srv2.run(reqs)
    close_server(srv2)
    cap_server = serve.summarize(done_c0)
    cap_sync = serve.summarize(done0)
    if rank != 0:
        return
    sv, sy = srv_main, sy_main
    line = {"metric": "serving: sustained updates/s and batch latency (resident R-MAT-22 + 64 tenants)",
            "value": sv["updates_per_s"], "unit": UNIT, "n_gpus": ws, "steps": len(reqs), "warmup": 0,
            "ms_per_step": round(sv["makespan_s"] / len(reqs) * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "resident R-MAT scale 22 + 64 R-MAT tenants (scales 14-18), 120 GB budget; "
                                   "Poisson arrivals, sizes log-uniform [100, 1M], 60/40 insert/delete, "
                                   "tenant Zipf(1.1), seed 5", "requests": len(reqs),
                       "load_vs_sync_capacity": args.load, "slots": 8, "coalescing": True,
                       "big_batch_priority_stream": ">= 50,000 edges", "reserved_batch_edges": 1_000_000,
                       "streams": "one own stream per tenant (+ one high-priority stream for big batches)"},
            "server": sv, "synchronous": sy, "latency_curve": curve,
            "capacity": {"server_updates_per_s": cap_server["updates_per_s"],
                         "synchronous_updates_per_s": cap_sync["updates_per_s"],
                         "server_over_sync": round(cap_server["updates_per_s"] / cap_sync["updates_per_s"], 3),
                         "what": "all requests queued at time 0"},
            "server_over_sync_updates_per_s": round(sv["updates_per_s"] / sy["updates_per_s"], 3),
            "coalesced_batches": coalesced, "evictions": evictions, "results_identical_to_alone": same}
    print(json.dumps(line), flush=True)


def cpu_baseline(g, steps, gpu_parents):
    """The serial oracle on the host cores, one step of the same trajectory
    (the first insert + delete batch from the initial state).  Its results
    are also compared with the GPU's parent arrays after the same two
    batches (True when both are bit-identical)."""
    import oracle
    keys, par = g.keys, g.parent
    t = 0.0
    applied = 0
    same = True
    for op in (0, 1):
        batch = steps[0][op][0]
        t0 = time.perf_counter()
        r = oracle.apply(g.n, keys, par, op, batch, want_keys=True)
        t += time.perf_counter() - t0
        applied += r.stats["applied"]
        keys, par = r.keys, r.parent
        same = same and bool(np.array_equal(par, gpu_parents[op]))
    return ({"value": round(applied / t, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"1 step (insert + delete, {len(steps[0][0][0])} edges each) of the same trajectory",
             "seconds": round(t, 3)}, same)


# ------------------------------------------------------------ reference arm

def run_reference(args, rank, ws):
    """The serial oracle as the reference arm: each step applies one batch of
    the trajectory (alternating insert / delete) on the host."""
    if rank != 0:
        return
    import oracle
    import workloads
    g, cfg = make_graph(args.workload)
    b = args.batch or cfg["batch"]
    tr = workloads.Trajectory(g, 5, tree_frac=cfg["tree_frac"], local=cfg["local"])
    keys, par = g.keys, g.parent
    t = 0.0
    applied = 0
    for s in range(args.warmup + args.steps):
        op = s % 2
        batch = tr.next_batch(op, b)
        t0 = time.perf_counter()
        r = oracle.apply(g.n, keys, par, op, batch, want_keys=True)
        dt = time.perf_counter() - t0
        keys, par = r.keys, r.parent
        tr.keys, tr.parent = keys, par
        if s >= args.warmup:
            t += dt
            applied += r.stats["applied"]
    v = round(applied / t, 1)
    line = {"impl": "reference",
            "metric": METRIC if args.workload == "rmat22" else f"updates/s ({args.workload}, {b}-update batches)",
            "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {**workload_config(args.workload, g, b), "parallelism": "single",
                       "reference_step": "one batch (alternating insert / delete) through the serial oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": f"{args.steps} batches of {b} edges, alternating insert/delete"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


ARGS = None


def main():
    global ARGS
    args = parse()
    ARGS = args
    rank, ws, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    elif args.workload == "batched256":
        run_batched(args, rank, ws, local)
    elif args.workload == "serving":
        run_serving(args, rank, ws, local)
    elif args.sweep:
        # batch-size sweep on one workload (latency per batch as b changes)
        for b in [int(x) for x in args.sweep.split(",") if x]:
            args.batch = b
            run_ours(args, rank, ws, local)
    else:
        run_ours(args, rank, ws, local)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
