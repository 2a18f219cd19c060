"""Serial CPU oracle for the D-RSF batch update (test infrastructure only).

This package is the plain, slow, obviously correct reference the GPU library
is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the GPU library never does.  It
shares no code with the GPU path.

All functions wrap ``oracle.c`` (compiled on first use with the system C
compiler) and follow the paper's definitions:

* :func:`apply` -- one batch update, Algorithm 1 with the deterministic
  readings listed in ``oracle.c`` (minimum-key replacement forest by Kruskal,
  smallest-root-id super-root, serial path reversal);
* :func:`check_forest` -- the exact checker that a parent array is a rooted
  spanning forest of a graph (D-RSF box, Section I; Section II-A);
* :func:`labels` -- connected-component labels, smallest vertex id
  (connectivity maintenance, Section I);
* :func:`representatives` -- rep[v], root of v's tree (Section II-A).

Every function here has pins in ``tests/test_oracle_*.py`` (brute force on
tiny graphs, closed forms, library routines); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

INSERT, DELETE = 0, 1

CHECK_OK = 0
CHECK_RANGE, CHECK_NOT_EDGE, CHECK_CYCLE, CHECK_ROOTS, CHECK_REACH = 1, 2, 3, 4, 5


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "batch_len", "self_loops", "duplicates", "ignored", "applied", "tree_cut", "pieces",
        "components", "cross", "replacement", "reversed", "m_out")]


@dataclass
class Result:
    parent: np.ndarray        # F'
    replacement: np.ndarray   # E_r keys, sorted
    keys: np.ndarray | None   # E(G') sorted, if requested
    stats: dict


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so next to it."""
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
            u64p, i32p, i64p = P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_int64)
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_labels.restype = ctypes.c_int
            lib.oracle_labels.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, i32p]
            lib.oracle_check_forest.restype = ctypes.c_int
            lib.oracle_check_forest.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, i32p]
            lib.oracle_representatives.restype = ctypes.c_int
            lib.oracle_representatives.argtypes = [ctypes.c_int32, i32p, i32p]
            lib.oracle_apply.restype = ctypes.c_int
            lib.oracle_apply.argtypes = [ctypes.c_int32, u64p, ctypes.c_int64, i32p, ctypes.c_int32, i32p,
                                         ctypes.c_int64, i32p, u64p, i64p, P(u64p), P(_Stats)]
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _keys(keys):
    return np.ascontiguousarray(keys, np.uint64)


def check_forest(n: int, keys: np.ndarray, parent: np.ndarray) -> int:
    """0 if `parent` is a rooted spanning forest of the graph, else the failed
    rule (CHECK_RANGE .. CHECK_REACH)."""
    keys = _keys(keys)
    parent = np.ascontiguousarray(parent, np.int32)
    rc = _load().oracle_check_forest(n, _p(keys, ctypes.c_uint64), len(keys), _p(parent, ctypes.c_int32))
    if rc < 0:
        raise MemoryError("oracle_check_forest")
    return rc


def labels(n: int, keys: np.ndarray) -> np.ndarray:
    """Smallest vertex id of each vertex's connected component."""
    keys = _keys(keys)
    out = np.empty(n, np.int32)
    rc = _load().oracle_labels(n, _p(keys, ctypes.c_uint64), len(keys), _p(out, ctypes.c_int32))
    if rc:
        raise ValueError(f"oracle_labels failed ({rc})")
    return out


def representatives(parent: np.ndarray) -> np.ndarray:
    """rep[v] = root of v's tree (parent must be an acyclic forest)."""
    parent = np.ascontiguousarray(parent, np.int32)
    out = np.empty(len(parent), np.int32)
    rc = _load().oracle_representatives(len(parent), _p(parent, ctypes.c_int32), _p(out, ctypes.c_int32))
    if rc:
        raise ValueError("invalid forest")
    return out


def apply(n: int, keys: np.ndarray, parent: np.ndarray, op: int, batch: np.ndarray,
          want_keys: bool = False) -> Result:
    """One D-RSF batch update (Algorithm 1).  Raises ValueError on invalid ids."""
    keys = _keys(keys)
    parent = np.ascontiguousarray(parent, np.int32)
    batch = np.ascontiguousarray(batch, np.int32).reshape(-1, 2)
    out = np.empty(n, np.int32)
    repl = np.empty(max(n, 1), np.uint64)
    nrepl = ctypes.c_int64(0)
    kp = ctypes.POINTER(ctypes.c_uint64)()
    st = _Stats()
    lib = _load()
    rc = lib.oracle_apply(n, _p(keys, ctypes.c_uint64), len(keys), _p(parent, ctypes.c_int32), op,
                          _p(batch, ctypes.c_int32), len(batch), _p(out, ctypes.c_int32),
                          _p(repl, ctypes.c_uint64), ctypes.byref(nrepl),
                          ctypes.byref(kp) if want_keys else None, ctypes.byref(st))
    if rc == -1:
        raise ValueError("invalid vertex id or parent array")
    if rc:
        raise MemoryError("oracle_apply")
    gk = None
    if want_keys:
        m2 = st.m_out
        gk = np.ctypeslib.as_array(kp, shape=(m2,)).copy() if m2 else np.zeros(0, np.uint64)
        lib.oracle_free(kp)
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return Result(out, repl[:nrepl.value].copy(), gk, stats)
