"""GB300 (sm_103a) dynamic rooted spanning forest: Python binding.

A thin ctypes layer over the C ABI in ``include/drsf.h`` (libdrsf.so, built
in-tree by :func:`build`).  It only marshals arguments: every step of the
batch update runs in the library's CUDA kernels.  PyTorch supplies device
memory (the library allocates through torch's caching allocator) and the
current CUDA stream.  There is no CPU fallback: if the library is missing the
import of the handle class fails loudly.

Example::

    import torch, paper_2607_20211_gb300 as drsf
    f = drsf.DynamicForest(n, edges_cuda_int32_mx2, parent_cuda_int32_n)
    f.insert(batch_cuda_int32_bx2)
    f.delete(other_batch)
    parent = f.parent()           # torch.int32 [n] on the device
    labels = f.labels()           # smallest vertex id of each component
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build_mod

INSERT, DELETE = 0, 1
DETERMINISTIC, VALIDATE, EULER_REVERSAL, REPL_SG, REPL_HS = 1, 2, 4, 8, 16

OK, EINVAL, ENOMEM, ECUDA, ENOT_FOREST, ETIMEOUT, EPOISONED = range(7)

LIB_PATH = _build_mod.LIB
_lib = None
_lock = threading.Lock()


class DRSFError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _load().drsf_error_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


class BatchStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "batch_len", "self_loops", "dropped", "applied", "tree_cut", "affected", "detached", "scanned",
        "candidates", "hook_rounds", "replacement", "rank_rounds", "active", "reversed", "mark_rounds",
        "jump_rounds", "edges", "overflow", "rebuilds", "jump_visits", "supergraph", "detach_levels",
        "detach_entries", "core_arcs")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


NUM_PHASES = 12


class BatchedClass(ctypes.Structure):
    """One size class of drsf_apply_batched: graphs with at most
    max_vertices vertices (and more than the previous class's), their block
    size, blocks per SM (0: as many as fit) and blocks per cluster (the
    group that updates one graph)."""
    _fields_ = [("max_vertices", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("cluster_blocks", ctypes.c_int32)]


# default size classes of the batched form:
# (max vertices, block threads, blocks per SM, blocks per cluster)
DEFAULT_CLASSES = ((8192, 256, 0, 1), (65536, 512, 0, 2), (2 ** 31 - 1, 1024, 0, 8))


class Profile(ctypes.Structure):
    _fields_ = [("ms", (ctypes.c_double * NUM_PHASES) * 2), ("launches", (ctypes.c_int64 * NUM_PHASES) * 2),
                ("batches", ctypes.c_int64 * 2)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_live_blocks: dict[int, torch.Tensor] = {}


def _torch_alloc(nbytes, stream, ctx):
    try:
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
    except RuntimeError:
        return None
    p = t.data_ptr()
    _live_blocks[p] = t
    return p


def _torch_free(ptr, stream, ctx):
    _live_blocks.pop(int(ptr or 0), None)


_c_alloc = _ALLOC_FN(_torch_alloc)
_c_free = _FREE_FN(_torch_free)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libdrsf.so for sm_103a (nvcc) if stale; return its path."""
    return _build_mod.build(force=force, verbose=verbose)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdrsf.so is not built ({LIB_PATH}); call paper_2607_20211_gb300.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        lib.drsf_set_allocator.restype = ctypes.c_int
        lib.drsf_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
        lib.drsf_create.restype = ctypes.c_int
        lib.drsf_create.argtypes = [i32, vp, i64, vp, u32, vp, P(vp)]
        for name in ("drsf_apply", "drsf_apply_host"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [vp, ctypes.c_int, vp, i64, vp]
        for name in ("drsf_parent", "drsf_labels"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [vp, vp, vp]
        lib.drsf_stats.restype = ctypes.c_int
        lib.drsf_stats.argtypes = [vp, P(BatchStats), vp]
        lib.drsf_sync.restype = ctypes.c_int
        lib.drsf_sync.argtypes = [vp, vp]
        lib.drsf_num_vertices.restype = i32
        lib.drsf_num_vertices.argtypes = [vp]
        lib.drsf_num_edges.restype = i64
        lib.drsf_num_edges.argtypes = [vp, vp]
        lib.drsf_export_edges.restype = ctypes.c_int
        lib.drsf_export_edges.argtypes = [vp, vp, i64, P(i64), vp]
        lib.drsf_destroy.restype = None
        lib.drsf_destroy.argtypes = [vp]
        lib.drsf_error_string.restype = ctypes.c_char_p
        lib.drsf_error_string.argtypes = [ctypes.c_int]
        lib.drsf_profile_start.restype = ctypes.c_int
        lib.drsf_profile_start.argtypes = [vp, i64]
        lib.drsf_profile_stop.restype = ctypes.c_int
        lib.drsf_profile_stop.argtypes = [vp, P(Profile), vp]
        lib.drsf_static_forest.restype = ctypes.c_int
        lib.drsf_static_forest.argtypes = [vp, vp, vp, P(i64), vp]
        lib.drsf_selftest_barrier_timeout.restype = ctypes.c_int
        lib.drsf_selftest_barrier_timeout.argtypes = [vp]
        lib.drsf_phase_name.restype = ctypes.c_char_p
        lib.drsf_phase_name.argtypes = [ctypes.c_int]
        lib.drsf_stream_create.restype = ctypes.c_int
        lib.drsf_stream_create.argtypes = [ctypes.c_int, P(vp)]
        lib.drsf_stream_destroy.restype = ctypes.c_int
        lib.drsf_stream_destroy.argtypes = [vp]
        lib.drsf_reserve.restype = ctypes.c_int
        lib.drsf_reserve.argtypes = [vp, i64, vp]
        lib.drsf_apply_batched.restype = ctypes.c_int
        lib.drsf_apply_batched.argtypes = [vp, ctypes.c_int, vp, i64, i32, vp, vp, vp, i32, vp]
        _lib = lib
        return lib


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _load()


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching
    allocator (the default for handles made by this module)."""
    lib = _load()
    if enable:
        st = lib.drsf_set_allocator(_c_alloc, _c_free, None)
    else:
        st = lib.drsf_set_allocator(_ALLOC_FN(), _FREE_FN(), None)
    if st:
        raise DRSFError(st, "drsf_set_allocator")


def selftest_barrier_timeout(stream=None) -> int:
    """Run the bounded-wait self-test; returns the status (ETIMEOUT expected)."""
    return int(_load().drsf_selftest_barrier_timeout(_stream_ptr(stream)))


class OwnStream:
    """A CUDA stream of its own (not from torch's stream pool, which hands
    the same few streams to every caller), usable as a torch stream through
    `.torch`; destroyed by close().  priority: a smaller number is a higher
    priority (clamped to the device's range)."""

    def __init__(self, priority: int = 0):
        p = ctypes.c_void_p()
        st = _load().drsf_stream_create(int(priority), ctypes.byref(p))
        if st:
            raise DRSFError(st, "drsf_stream_create")
        self.ptr = p.value
        self.torch = torch.cuda.ExternalStream(self.ptr)

    def close(self) -> None:
        if self.ptr:
            torch.cuda.synchronize()
            _load().drsf_stream_destroy(self.ptr)
            self.ptr = None


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_i32(t: torch.Tensor, name: str, cols: int | None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.int32:
        raise TypeError(f"{name} must be int32")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols) and t.numel() != 0:
        raise ValueError(f"{name} must have shape [k, {cols}]")
    return t.contiguous()


class DynamicForest:
    """A rooted spanning forest of an undirected graph, kept on one GPU and
    updated batch by batch (D-RSF, Algorithm 1)."""

    def __init__(self, n: int, edges: torch.Tensor, parent: torch.Tensor, flags: int = DETERMINISTIC,
                 stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        lib = _load()
        if torch_allocator:
            use_torch_allocator(True)
        edges = _dev_i32(edges, "edges", 2)
        parent = _dev_i32(parent, "parent", None)
        if parent.numel() != n:
            raise ValueError("parent must have n entries")
        self._n = int(n)
        self._stream = stream
        h = ctypes.c_void_p()
        st = lib.drsf_create(self._n, edges.data_ptr() if edges.numel() else None, int(edges.shape[0]) if
                             edges.numel() else 0, parent.data_ptr(), flags, _stream_ptr(stream), ctypes.byref(h))
        if torch_allocator:
            use_torch_allocator(False)
        if st:
            raise DRSFError(st, "drsf_create")
        self._h = h
        self._keep = (edges, parent)

    # -- updates ----------------------------------------------------------
    def apply(self, op: int, batch: torch.Tensor) -> None:
        """Enqueue one batch (insert or delete) on the handle's stream."""
        batch = _dev_i32(batch, "batch", 2)
        st = _lib.drsf_apply(self._h, op, batch.data_ptr() if batch.numel() else None,
                             int(batch.shape[0]) if batch.numel() else 0, _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_apply")

    def apply_host(self, op: int, batch) -> None:
        """Same as apply, with the batch in host memory (numpy int32 [b, 2] or
        a CPU tensor); the library stages it to the device."""
        t = torch.as_tensor(batch, dtype=torch.int32).contiguous()
        if t.numel() and (t.dim() != 2 or t.shape[1] != 2):
            raise ValueError("batch must have shape [b, 2]")
        st = _lib.drsf_apply_host(self._h, op, t.data_ptr() if t.numel() else None,
                                  int(t.shape[0]) if t.numel() else 0, _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_apply_host")

    def apply_batched(self, op: int, batch: torch.Tensor, vertex_offsets, batch_offsets,
                      classes=DEFAULT_CLASSES) -> None:
        """Batched form: the handle holds the disjoint union of independent
        graphs (graph g owns vertices vertex_offsets[g] .. vertex_offsets[g+1]
        and batch rows batch_offsets[g] .. batch_offsets[g+1]); persistent
        per-graph kernels apply every graph's slice.  `classes` is a sequence
        of (max_vertices, block_threads, blocks_per_sm[, cluster_blocks])
        size classes."""
        import numpy as np
        batch = _dev_i32(batch, "batch", 2)
        vo = np.ascontiguousarray(vertex_offsets, np.int64)
        bo = np.ascontiguousarray(batch_offsets, np.int64)
        if vo.shape != bo.shape or vo.ndim != 1 or len(vo) < 2:
            raise ValueError("vertex_offsets and batch_offsets must be 1-D of the same length G + 1")
        rows = [tuple(c) + (1,) * (4 - len(c)) for c in classes]
        cl = (BatchedClass * len(rows))(*[BatchedClass(*(int(x) for x in r)) for r in rows])
        st = _lib.drsf_apply_batched(self._h, op, batch.data_ptr() if batch.numel() else None,
                                     int(batch.shape[0]) if batch.numel() else 0, len(vo) - 1,
                                     vo.ctypes.data, bo.ctypes.data, ctypes.cast(cl, ctypes.c_void_p),
                                     len(classes), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_apply_batched")

    def reserve(self, max_batch: int) -> None:
        """Size the per-batch buffers for batches of up to max_batch edges
        now (no allocation or synchronisation for them later)."""
        st = _lib.drsf_reserve(self._h, int(max_batch), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_reserve")

    def insert(self, batch: torch.Tensor) -> None:
        self.apply(INSERT, batch)

    def delete(self, batch: torch.Tensor) -> None:
        self.apply(DELETE, batch)

    # -- results ----------------------------------------------------------
    def parent(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty(self._n, dtype=torch.int32, device="cuda") if out is None else out
        st = _lib.drsf_parent(self._h, out.data_ptr(), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_parent")
        return out

    def labels(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = torch.empty(self._n, dtype=torch.int32, device="cuda") if out is None else out
        st = _lib.drsf_labels(self._h, out.data_ptr(), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_labels")
        return out

    def stats(self) -> dict:
        s = BatchStats()
        st = _lib.drsf_stats(self._h, ctypes.byref(s), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_stats")
        return s.as_dict()

    def sync(self) -> None:
        st = _lib.drsf_sync(self._h, _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_sync")

    @property
    def n(self) -> int:
        return self._n

    def num_edges(self) -> int:
        return int(_lib.drsf_num_edges(self._h, _stream_ptr(self._stream)))

    def export_edges(self) -> torch.Tensor:
        m = self.num_edges()
        out = torch.empty((max(m, 1), 2), dtype=torch.int32, device="cuda")
        got = ctypes.c_int64(0)
        st = _lib.drsf_export_edges(self._h, out.data_ptr(), out.shape[0], ctypes.byref(got),
                                    _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_export_edges")
        return out[:got.value]

    def static_forest(self, with_levels: bool = False):
        """A rooted spanning forest of the current graph rebuilt from scratch
        (components + multi-source BFS from their minima); returns
        (parent, labels[, levels]) as device tensors."""
        par = torch.empty(self._n, dtype=torch.int32, device="cuda")
        lab = torch.empty(self._n, dtype=torch.int32, device="cuda")
        lv = ctypes.c_int64(0)
        st = _lib.drsf_static_forest(self._h, par.data_ptr(), lab.data_ptr(),
                                     ctypes.byref(lv) if with_levels else None, _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_static_forest")
        return (par, lab, lv.value) if with_levels else (par, lab)

    def profile_start(self, max_batches: int) -> None:
        """Start per-phase CUDA-event timing of the next batches."""
        st = _lib.drsf_profile_start(self._h, int(max_batches))
        if st:
            raise DRSFError(st, "drsf_profile_start")

    def profile_stop(self) -> dict:
        """Stop timing; {"insert"|"delete": {phase: (ms, launches)}} plus
        the number of batches of each kind under "batches"."""
        p = Profile()
        st = _lib.drsf_profile_stop(self._h, ctypes.byref(p), _stream_ptr(self._stream))
        if st:
            raise DRSFError(st, "drsf_profile_stop")
        out = {}
        for o, name in ((0, "insert"), (1, "delete")):
            out[name] = {_lib.drsf_phase_name(i).decode(): (p.ms[o][i], p.launches[o][i])
                         for i in range(NUM_PHASES)}
        out["batches"] = {"insert": p.batches[0], "delete": p.batches[1]}
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.drsf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
