"""Schedule autotuner of the batched form (drsf_apply_batched).

The persistent per-graph kernels put graphs into size classes by vertex
count; each class has its own block size, blocks per SM and cluster size
(the blocks that update one graph together).  The tuner picks them per
(size class, operation) by timing candidate schedules on the
caller's own workload: every trial starts from the same state (a fresh
handle built from the same edge list and parent array) and applies the same
union batch, so trials differ only in the schedule.  Classes are tuned one
after another with the others held at their current best (coordinate
descent), insert and delete separately.  The result is cached in a JSON file
keyed by size class and operation, together with a signature of the
workload and the GPU, and reused while both match.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import DEFAULT_CLASSES, DynamicForest, INSERT, DELETE

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batched.json")
# (block threads, blocks per SM (0 = as many as fit), blocks per cluster)
CANDIDATES = ((256, 0, 1), (512, 0, 1), (1024, 0, 1), (1024, 1, 1), (256, 0, 2), (512, 0, 2), (1024, 0, 2),
              (512, 0, 4), (1024, 0, 4), (512, 0, 8), (1024, 0, 8), (1024, 0, 16))
OPS = {INSERT: "insert", DELETE: "delete"}


def signature(vertex_offsets, gpu_name: str | None = None) -> str:
    """Workload + device signature: graph count, size histogram per class, GPU."""
    vo = np.asarray(vertex_offsets, np.int64)
    sizes = np.diff(vo)
    hist = [int(np.sum((sizes > lo) & (sizes <= hi))) for lo, hi in
            zip((0,) + tuple(c[0] for c in DEFAULT_CLASSES[:-1]), tuple(c[0] for c in DEFAULT_CLASSES))]
    name = gpu_name or (torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu")
    return f"G={len(sizes)};n={int(vo[-1] - vo[0])};classes={hist};gpu={name}"


def load(sig: str, path: str = CACHE):
    """The cached schedules {op: classes} for this signature, or None."""
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("signature") != sig:
        return None
    out = {}
    for op, name in OPS.items():
        rows = [d["schedule"].get(f"class<={c[0]}/{name}") for c in DEFAULT_CLASSES]
        if any(r is None for r in rows):
            return None
        out[op] = tuple((c[0], int(r["block_threads"]), int(r["blocks_per_sm"]), int(r["cluster_blocks"]))
                        for c, r in zip(DEFAULT_CLASSES, rows))
    return out


def _time(n, edges, parent, op, batch, vo, bo, classes):
    """Device time (ms) of one apply_batched from the given state.  An empty
    batch with the same graphs and classes goes first, so the launch
    sequence is captured before the timed call (same capture key)."""
    f = DynamicForest(n, edges, parent)
    try:
        empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
        f.apply_batched(op, empty, vo, np.zeros_like(bo), classes)
        f.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f.apply_batched(op, batch, vo, bo, classes)
        e1.record()
        f.sync()
        return e0.elapsed_time(e1)
    finally:
        f.close()


def tune(n, states, vertex_offsets, batches, path: str = CACHE, log=None):
    """Pick the schedule per (size class, op).

    states:  {op: (edges int32[m,2] cuda, parent int32[n] cuda)}, the state
             before that op's batch
    batches: {op: (union batch int32[b,2] cuda, batch_offsets int64[G+1])}
    Returns {op: classes} and writes the cache."""
    vo = np.asarray(vertex_offsets, np.int64)
    sig = signature(vo)
    result, table = {}, {}
    for op, name in OPS.items():
        edges, parent = states[op]
        batch, bo = batches[op]
        cur = [list(c) for c in DEFAULT_CLASSES]
        base = _time(n, edges, parent, op, batch, vo, bo, tuple(map(tuple, cur)))
        for ci in range(len(cur)):
            best_t, best_c = base, tuple(cur[ci][1:])
            for cand in CANDIDATES:
                trial = [list(c) for c in cur]
                trial[ci][1:] = list(cand)
                t = _time(n, edges, parent, op, batch, vo, bo, tuple(map(tuple, trial)))
                if log:
                    log(f"tune {name} class<={cur[ci][0]} threads={cand[0]} per_sm={cand[1]} cluster={cand[2]}: "
                        f"{t:.3f} ms")
                if t < best_t:
                    best_t, best_c = t, tuple(cand)
            cur[ci][1:] = list(best_c)
            base = best_t
        result[op] = tuple(map(tuple, cur))
        for c in cur:
            table[f"class<={c[0]}/{name}"] = {"block_threads": c[1], "blocks_per_sm": c[2], "cluster_blocks": c[3]}
        table[f"ms/{name}"] = round(base, 4)
    json.dump({"signature": sig, "schedule": table,
               "candidates": [list(c) for c in CANDIDATES],
               "what": "per size class (max vertices) and op: block threads, blocks per SM and blocks per cluster of "
                       "the persistent per-graph kernel, by coordinate descent over timed trials from one fixed state"},
              open(path, "w"), indent=1)
    return result
