"""Parallel oracle checks of long GPU trajectories (test infrastructure).

A trajectory is checked batch by batch: batch i must take the oracle from
state i-1 to the GPU's state i (parent array bit for bit, labels, the exact
checker, the counters).  The oracle's start state for batch i is the GPU's
state i-1 (its parent array; the edge set follows from the batches), so the
checks of different batches are independent and run side by side in a pool
of processes; by induction over i they are the same check as one serial
oracle run along the whole trajectory.

The pool uses the ``spawn`` start method (a forked child of a process that
has touched CUDA can hang).  Workers exchange arrays through ``.npy`` files
in a temporary directory, so only paths cross the process boundary.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

_POOL = None


def _memory_gb() -> float:
    """Memory this process may still use: MemAvailable, capped by a cgroup
    limit when one is set."""
    avail = 64.0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    try:
        lim = open("/sys/fs/cgroup/memory.max").read().strip()
        if lim != "max":
            used = int(open("/sys/fs/cgroup/memory.current").read())
            avail = min(avail, (int(lim) - used) / 2 ** 30)
    except (OSError, ValueError):
        pass
    return avail


def pool():
    """The shared process pool (created on first use, spawn start method):
    one worker per spare core, at most one per 6 GB of free memory (an
    oracle run on R-MAT scale 22 holds about 4 GB)."""
    global _POOL
    if _POOL is None:
        workers = max(1, min(15, (os.cpu_count() or 2) - 1, int(_memory_gb() // 6)))
        _POOL = mp.get_context("spawn").Pool(workers)
    return _POOL


def shutdown():
    global _POOL
    if _POOL is not None:
        _POOL.close()
        _POOL.join()
        _POOL = None


def _check(task):
    """Worker: one batch of a trajectory against the oracle.  Returns None
    when everything matches, else a description of the first mismatch."""
    import oracle
    import workloads
    n = task["n"]
    keys = np.load(task["keys0"])
    for path, op in task["history"]:          # E(G) before this batch
        keys = workloads.apply_keys(keys, np.load(path), op)
    par = np.load(task["parent_in"]) if task["parent_in"] else np.load(task["parent0"])
    batch = np.load(task["batch"])
    got = np.load(task["parent_out"])
    ref = oracle.apply(n, keys, par, task["op"], batch, want_keys=True)
    tag = f"batch {task['index']} (op {task['op']}, {len(batch)} edges)"
    if not np.array_equal(got, ref.parent):
        bad = np.nonzero(got != ref.parent)[0]
        return (f"{tag}: parent differs at {len(bad)} vertices, first {bad[:8].tolist()}: "
                f"gpu {got[bad[:8]].tolist()} oracle {ref.parent[bad[:8]].tolist()}")
    rc = oracle.check_forest(n, ref.keys, got)
    if rc:
        return f"{tag}: exact checker rejects the forest (rule {rc})"
    st = task["stats"]
    want = {} if st is None else {"applied": ref.stats["applied"], "self_loops": ref.stats["self_loops"],
            "dropped": ref.stats["duplicates"] + ref.stats["ignored"], "tree_cut": ref.stats["tree_cut"],
            "replacement": ref.stats["replacement"], "edges": ref.stats["m_out"]}
    for k, v in want.items():
        if st[k] != v:
            return f"{tag}: counter {k} gpu {st[k]} oracle {v}"
    if task.get("labels_out"):
        lab = np.load(task["labels_out"])
        if not np.array_equal(lab, oracle.labels(n, ref.keys)):
            return f"{tag}: labels differ from the oracle's component minima"
    return None


class TrajectoryCheck:
    """Collects the GPU side of a trajectory and checks it in the pool."""

    def __init__(self, n: int, keys0: np.ndarray, parent0: np.ndarray):
        self.dir = tempfile.mkdtemp(prefix="drsf_parity_")
        self.n = n
        self.keys0 = os.path.join(self.dir, "keys0.npy")
        self.parent0 = os.path.join(self.dir, "parent_initial.npy")
        np.save(self.keys0, np.ascontiguousarray(keys0, np.uint64))
        np.save(self.parent0, np.ascontiguousarray(parent0, np.int32))
        self.history = []
        self.prev_parent = None
        self.pending = []

    def add(self, op: int, batch: np.ndarray, parent_out: np.ndarray, stats: dict | None,
            labels_out: np.ndarray | None = None):
        """Queue the check of one batch: `parent_out`, `labels_out` and the
        counters `stats` (None: not compared) are the GPU's after `batch`."""
        i = len(self.history)
        bpath = os.path.join(self.dir, f"batch{i}.npy")
        ppath = os.path.join(self.dir, f"parent_after{i}.npy")
        np.save(bpath, np.ascontiguousarray(batch, np.int32).reshape(-1, 2))
        np.save(ppath, np.ascontiguousarray(parent_out, np.int32))
        lpath = None
        if labels_out is not None:
            lpath = os.path.join(self.dir, f"labels{i}.npy")
            np.save(lpath, np.ascontiguousarray(labels_out, np.int32))
        task = {"n": self.n, "keys0": self.keys0, "parent0": self.parent0, "history": list(self.history),
                "parent_in": self.prev_parent, "batch": bpath, "op": int(op), "parent_out": ppath,
                "labels_out": lpath, "index": i,
                "stats": None if stats is None else {k: int(v) for k, v in stats.items()}}
        self.pending.append(pool().apply_async(_check, (task,)))
        self.history.append((bpath, int(op)))
        self.prev_parent = ppath

    def result(self):
        """Wait for every check; raise AssertionError on the first mismatch."""
        try:
            errs = [r.get(timeout=1500) for r in self.pending]
        finally:
            shutil.rmtree(self.dir, ignore_errors=True)
        errs = [e for e in errs if e]
        if errs:
            raise AssertionError("; ".join(errs[:3]))
        return len(self.pending)
