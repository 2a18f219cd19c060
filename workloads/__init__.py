"""Seeded synthetic workloads for the dynamic rooted spanning forest update.

Input plumbing only: graphs (Erdos-Renyi, R-MAT with the Graph500 initiator,
road-like grids), the initial FIFO-BFS forest and update batches.  Both the
serial oracle's tests and the GPU library's tests and benchmark draw their
inputs from here; the module contains none of the update method's arithmetic.
The generators stand in for the paper's datasets (Section V, Table III),
which are not available offline.

The C core (``gen.c``) is compiled on first use with the system C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_gen.so")
_lock = threading.Lock()
_lib = None

RMAT_GRAPH500 = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile gen.c into _gen.so next to it (portable flags, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            u64p, i32p = P(ctypes.c_uint64), P(ctypes.c_int32)
            lib.gen_free.argtypes = [ctypes.c_void_p]
            lib.gen_er.restype = ctypes.c_int64
            lib.gen_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, P(u64p)]
            lib.gen_rmat.restype = ctypes.c_int64
            lib.gen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P(u64p)]
            lib.gen_grid.restype = ctypes.c_int64
            lib.gen_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64,
                                     ctypes.c_uint64, P(u64p)]
            lib.gen_bfs_forest.restype = ctypes.c_int
            lib.gen_bfs_forest.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, i32p]
            lib.gen_insert_batch.restype = ctypes.c_int
            lib.gen_insert_batch.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gen_delete_batch.restype = ctypes.c_int64
            lib.gen_delete_batch.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, i32p, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gen_apply_keys.restype = ctypes.c_int64
            lib.gen_apply_keys.argtypes = [u64p, ctypes.c_int64, i32p, ctypes.c_int64, ctypes.c_int32,
                                           P(u64p)]
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _take(ptr, count):
    lib = _load()
    if count < 0:
        raise MemoryError("generator allocation failed")
    if count == 0:
        if ptr:
            lib.gen_free(ptr)
        return np.zeros(0, np.uint64)
    arr = np.ctypeslib.as_array(ptr, shape=(count,)).copy()
    lib.gen_free(ptr)
    return arr


def _prob32(p: float) -> int:
    return min(int(round(p * 2 ** 32)), 2 ** 32 - 1)


def er(n: int, m: int, seed: int) -> np.ndarray:
    """G(n, m): m distinct non-loop pairs; sorted uint64 keys (min<<32|max)."""
    ptr = ctypes.POINTER(ctypes.c_uint64)()
    c = _load().gen_er(n, m, seed, ctypes.byref(ptr))
    return _take(ptr, c)


def rmat(scale: int, edge_factor: int, seed: int, n: int | None = None,
         abc=RMAT_GRAPH500) -> np.ndarray:
    """R-MAT keys over n vertices (default 2^scale), ids permuted."""
    a, b, c = abc
    ptr = ctypes.POINTER(ctypes.c_uint64)()
    cnt = _load().gen_rmat(scale, n or 0, edge_factor, _prob32(a), _prob32(b), _prob32(c), seed,
                           ctypes.byref(ptr))
    return _take(ptr, cnt)


def grid(W: int, H: int, seed: int, keep: float = 0.6, shortcut_frac: float = 0.001) -> np.ndarray:
    """W x H grid, ids y*W+x, each 4-neighbour edge kept with prob `keep`,
    plus round(shortcut_frac * W * H) uniform shortcuts."""
    ptr = ctypes.POINTER(ctypes.c_uint64)()
    cnt = _load().gen_grid(W, H, _prob32(keep), int(round(shortcut_frac * W * H)), seed,
                           ctypes.byref(ptr))
    return _take(ptr, cnt)


def bfs_forest(n: int, keys: np.ndarray) -> np.ndarray:
    """FIFO BFS forest from each component's smallest id (parent[root]=root)."""
    keys = np.ascontiguousarray(keys, np.uint64)
    parent = np.empty(n, np.int32)
    if _load().gen_bfs_forest(n, _p(keys, ctypes.c_uint64), len(keys), _p(parent, ctypes.c_int32)):
        raise MemoryError("bfs_forest")
    return parent


def insert_batch(n: int, keys: np.ndarray, b: int, seed: int, W: int = 0, local: int = 0) -> np.ndarray:
    """b distinct new pairs not in `keys` (sorted), random orientation, int32[b, 2].
    With local > 0, the second endpoint lies within `local` cells on a W-wide grid."""
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty((b, 2), np.int32)
    rc = _load().gen_insert_batch(n, _p(keys, ctypes.c_uint64), len(keys), b, W, local, seed,
                                  _p(out, ctypes.c_int32))
    if rc:
        raise RuntimeError(f"insert_batch failed ({rc})")
    return out


def delete_batch(n: int, keys: np.ndarray, parent: np.ndarray, b: int, tree_frac: float,
                 seed: int) -> np.ndarray:
    """b distinct existing edges, about tree_frac of them tree edges of `parent`."""
    keys = np.ascontiguousarray(keys, np.uint64)
    parent = np.ascontiguousarray(parent, np.int32)
    out = np.empty((max(b, 0), 2), np.int32)
    c = _load().gen_delete_batch(n, _p(keys, ctypes.c_uint64), len(keys), _p(parent, ctypes.c_int32), b,
                                 int(round(tree_frac * 1000)), seed, _p(out, ctypes.c_int32))
    if c < 0:
        raise MemoryError("delete_batch")
    return out[:c].copy()


def apply_keys(keys: np.ndarray, batch: np.ndarray, op: int) -> np.ndarray:
    """Sorted key set after inserting (op=0) or deleting (op=1) `batch`."""
    keys = np.ascontiguousarray(keys, np.uint64)
    batch = np.ascontiguousarray(batch, np.int32).reshape(-1, 2)
    ptr = ctypes.POINTER(ctypes.c_uint64)()
    c = _load().gen_apply_keys(_p(keys, ctypes.c_uint64), len(keys), _p(batch, ctypes.c_int32), len(batch),
                               op, ctypes.byref(ptr))
    return _take(ptr, c)


def keys_to_edges(keys: np.ndarray) -> np.ndarray:
    """uint64 keys -> int32[m, 2] (min, max)."""
    keys = np.asarray(keys, np.uint64)
    e = np.empty((len(keys), 2), np.int32)
    e[:, 0] = (keys >> np.uint64(32)).astype(np.int32)
    e[:, 1] = (keys & np.uint64(0xFFFFFFFF)).astype(np.int32)
    return e


def edges_to_keys(edges: np.ndarray) -> np.ndarray:
    """int32[m, 2] -> sorted unique uint64 keys, self-loops dropped."""
    e = np.asarray(edges, np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    lo = np.minimum(e[:, 0], e[:, 1]).astype(np.uint64)
    hi = np.maximum(e[:, 0], e[:, 1]).astype(np.uint64)
    return np.unique((lo << np.uint64(32)) | hi)


# ----------------------------------------------------------------- configs

class Graph:
    """A generated graph: n, sorted keys, initial BFS forest, generator info."""

    def __init__(self, name: str, n: int, keys: np.ndarray, W: int = 0):
        self.name, self.n, self.keys, self.W = name, n, keys, W
        self.parent = bfs_forest(n, keys)

    @property
    def m(self) -> int:
        return len(self.keys)

    def edges(self) -> np.ndarray:
        return keys_to_edges(self.keys)


def er_graph(n: int = 20_000, m: int = 25_000, seed: int = 1) -> Graph:
    """Erdos-Renyi G(n, m) (small configuration: n=20,000, m=25,000, seed 1)."""
    return Graph(f"er-{n}-{m}", n, er(n, m, seed))


def rmat_graph(scale: int = 20, edge_factor: int = 16, seed: int = 2, n: int | None = None) -> Graph:
    """R-MAT(scale, edge_factor), Graph500 initiator, ids permuted."""
    nn = n or (1 << scale)
    return Graph(f"rmat-{scale}-{edge_factor}", nn, rmat(scale, edge_factor, seed, n))


def grid_graph(W: int = 4096, H: int = 4096, seed: int = 3, keep: float = 0.6,
               shortcut_frac: float = 0.001) -> Graph:
    """Road-like grid: W x H, edges kept with p=keep, plus shortcut_frac*n shortcuts."""
    return Graph(f"grid-{W}x{H}", W * H, grid(W, H, seed, keep, shortcut_frac), W=W)


class Trajectory:
    """Alternating insert/delete batches on an evolving graph.

    Batches are generated from the *current* graph and forest, which the
    caller advances with :meth:`advance` (the forest comes from whichever
    implementation is being driven)."""

    def __init__(self, g: Graph, seed: int, tree_frac: float = 0.5, local: int = 0):
        self.n, self.keys, self.parent, self.W = g.n, g.keys.copy(), g.parent.copy(), g.W
        self.seed, self.tree_frac, self.local, self.step = seed, tree_frac, local, 0

    def next_batch(self, op: int, b: int) -> np.ndarray:
        s = (self.seed << 20) + self.step
        self.step += 1
        if op == 0:
            return insert_batch(self.n, self.keys, b, s, self.W, self.local)
        return delete_batch(self.n, self.keys, self.parent, b, self.tree_frac, s)

    def advance(self, batch: np.ndarray, op: int, parent: np.ndarray) -> None:
        self.keys = apply_keys(self.keys, batch, op)
        self.parent = np.ascontiguousarray(parent, np.int32).copy()


# ------------------------------------------------------- many small graphs

def batched_graphs(count: int = 256, seed: int = 4, n_lo: int = 1_000, n_hi: int = 256_000):
    """Independent graphs with n log-uniform in [n_lo, n_hi] and average
    degree uniform in [4, 16]; even indices Erdos-Renyi, odd R-MAT (sampled
    at scale ceil(log2 n), endpoints >= n dropped after the permutation)."""
    import math
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        deg = float(rng.uniform(4.0, 16.0))
        gseed = (seed << 16) + i
        if i % 2 == 0:
            m = int(n * deg / 2)
            keys = er(n, min(m, n * (n - 1) // 2), gseed)
            out.append(Graph(f"er-{n}", n, keys))
        else:
            scale = max(1, math.ceil(math.log2(n)))
            N = 1 << scale
            ef = max(1, int(round(deg * N / (2.0 * n))))
            keys = rmat(scale, ef, gseed, n=n)
            out.append(Graph(f"rmat-{n}", n, keys))
    return out


class Union:
    """Disjoint union of graphs with vertex-id offsets: one instance whose
    update is the per-graph updates side by side."""

    def __init__(self, graphs):
        self.graphs = graphs
        self.offsets = np.zeros(len(graphs) + 1, np.int64)
        for i, g in enumerate(graphs):
            self.offsets[i + 1] = self.offsets[i] + g.n
        self.n = int(self.offsets[-1])
        if self.n >= 2 ** 31:
            raise ValueError("union too large for int32 ids")
        ks, ps = [], []
        for g, off in zip(graphs, self.offsets[:-1]):
            o = np.uint64(off)
            lo = (g.keys >> np.uint64(32)) + o
            hi = (g.keys & np.uint64(0xFFFFFFFF)) + o
            ks.append((lo << np.uint64(32)) | hi)
            ps.append(g.parent.astype(np.int64) + off)
        self.keys = np.sort(np.concatenate(ks)) if ks else np.zeros(0, np.uint64)
        self.parent = np.concatenate(ps).astype(np.int32)

    def shift(self, i: int, batch: np.ndarray) -> np.ndarray:
        return (np.asarray(batch, np.int64) + self.offsets[i]).astype(np.int32)

    def split(self, arr: np.ndarray):
        """Per-graph slices of a union vertex array, ids shifted back."""
        return [(arr[self.offsets[i]:self.offsets[i + 1]].astype(np.int64) - self.offsets[i]).astype(np.int32)
                for i in range(len(self.graphs))]


def batched_budgets(graphs, seed: int = 4, lo: float = 0.01, hi: float = 0.10, ins_frac: float = 0.6):
    """Per graph one update budget of lo..hi of its m edges, split into an
    insert batch size (ins_frac) and a delete batch size (the rest)."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for g in graphs:
        budget = max(2, int(round(rng.uniform(lo, hi) * max(g.m, 1))))
        b_ins = max(1, int(round(ins_frac * budget)))
        out.append((b_ins, max(1, budget - b_ins)))
    return out
