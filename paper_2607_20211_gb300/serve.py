"""Serving loop: many resident graphs, update batches arriving over time.

Continuous batching over the C ABI:

* every admitted tenant (graph + forest) is a library handle with its own
  CUDA stream, so batches of different tenants run on the device at the
  same time;
* a tenant's requests are applied in arrival order, one batch in flight per
  tenant; requests that arrive while earlier ones are on the GPU wait in the
  tenant's queue and are admitted as soon as a slot and the tenant are free;
* consecutive queued requests of the same operation for one tenant are
  coalesced into one batch (insert B1 then insert B2 changes the graph as
  insert B1 + B2 does; the forest is the one the coalesced batch gives);
* tenants are admitted under a device-memory budget: a tenant that is not
  resident is created on demand, and idle tenants are evicted to host memory
  (edge list + parent array, re-created later with the same forest) when the
  budget would be exceeded; the storage a handle grows while it applies
  batches is charged to its tenant as it happens;
* scheduling is size-aware: a batch of at least `big_batch` edges (one that
  fills the device by itself) is admitted ahead of small ones and runs on
  the tenant's high-priority stream, so the block scheduler serves its
  kernels first and small tenants' batches fill the SMs it leaves idle
  (with exclusive_big, a big batch instead waits for the device to drain
  and runs alone: measured worse for both p50 and p99);
* every tenant has streams of its own (a framework's stream pool would let
  two tenants share a stream and queue behind each other), and its
  per-batch buffers are sized up front (reserve_edges), so no allocation
  or synchronisation inside one tenant's apply stalls the others;
* completions are found by querying the in-flight batches' CUDA events
  (measured: waiter threads blocking on the events delayed completions by
  Python thread switches and served no better than one batch at a time).

Every applied (coalesced) batch is logged per tenant, so any tenant's result
can be reproduced by applying its log alone.  Coalescing consecutive
same-operation requests keeps each tenant's labels and the validity of its
forest, but not necessarily the parent array that applying the requests one
by one would give (a merged batch may pick other replacement edges).
"""
from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import DETERMINISTIC, DynamicForest, OwnStream


@dataclass
class Request:
    rid: int
    tenant: int
    op: int
    batch: np.ndarray          # int32 [b, 2], host memory
    t_arrive: float = 0.0      # seconds from the start of the run


@dataclass
class Done:
    rid: int
    tenant: int
    t_arrive: float
    t_done: float
    updates: int


@dataclass
class Tenant:
    tid: int
    n: int
    edges: np.ndarray | None     # host state while not resident
    parent: np.ndarray | None
    handle: DynamicForest | None = None
    stream: torch.cuda.Stream | None = None    # the tenant's own stream (not a pooled one)
    fast: torch.cuda.Stream | None = None      # its high-priority stream for big batches
    own: list = field(default_factory=list)    # the OwnStream objects behind them
    bytes: int = 0
    last_used: float = 0.0
    queue: collections.deque = field(default_factory=collections.deque)
    inflight: list | None = None
    event: torch.cuda.Event | None = None
    log: list = field(default_factory=list)   # applied (op, batch) in order


class Server:
    """Continuous-batching server for D-RSF tenants on one GPU."""

    def __init__(self, budget_bytes: int = 120 << 30, slots: int = 8, coalesce: bool = True,
                 max_coalesce_edges: int = 2_000_000, flags: int = DETERMINISTIC, big_batch: int = 50_000,
                 exclusive_big: bool = False, priority_big: bool = True, reserve_edges: int = 0):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.coalesce = coalesce
        self.max_coalesce = int(max_coalesce_edges)
        self.flags = flags
        self.big_batch = int(big_batch)
        self.exclusive_big = exclusive_big
        self.priority_big = priority_big
        self.reserve_edges = int(reserve_edges or 0)
        self.tenants: dict[int, Tenant] = {}
        self.used = 0
        self.evictions = 0
        self.admissions = 0

    # -- tenants ------------------------------------------------------------
    def add_tenant(self, tid: int, n: int, edges: np.ndarray, parent: np.ndarray) -> None:
        self.tenants[tid] = Tenant(tid, int(n), np.ascontiguousarray(edges, np.int32).reshape(-1, 2),
                                   np.ascontiguousarray(parent, np.int32))

    def _estimate(self, t: Tenant) -> int:
        m = len(t.edges) if t.edges is not None else 0
        # per-vertex work arrays + CSR with slack + edge index + candidates,
        # plus the reserved per-batch buffers (work lists, pair table, staging)
        return 120 * t.n + 60 * m + 96 * self.reserve_edges + (8 << 20)

    def _admit(self, t: Tenant) -> bool:
        if t.handle is not None:
            return True
        need = self._estimate(t)
        while self.used + need > self.budget:
            idle = [u for u in self.tenants.values() if u.handle is not None and u.inflight is None]
            if not idle:
                return False
            self._evict(min(idle, key=lambda u: u.last_used))
        if t.stream is None:
            # streams of the tenant's own (a normal one and a high-priority
            # one for big batches): streams from torch's pool are shared
            # round-robin, and two tenants on one stream would queue behind
            # each other
            own, fast = OwnStream(0), OwnStream(-100)
            t.own += [own, fast]
            t.stream, t.fast = own.torch, fast.torch
        before = torch.cuda.memory_allocated()
        with torch.cuda.stream(t.stream):
            t.handle = DynamicForest(t.n, torch.from_numpy(t.edges).cuda(), torch.from_numpy(t.parent).cuda(),
                                     flags=self.flags, stream=t.stream)
            # per-batch buffers for the largest expected batch up front: an
            # allocation or a synchronisation inside one tenant's apply would
            # stall the loop and with it every tenant in flight
            if self.reserve_edges:
                t.handle.reserve(self.reserve_edges)
        t.bytes = max(torch.cuda.memory_allocated() - before, need)
        self.used += t.bytes
        t.edges = t.parent = None
        self.admissions += 1
        return True

    def _evict(self, t: Tenant) -> None:
        with torch.cuda.stream(t.stream):
            t.edges = t.handle.export_edges().cpu().numpy()
            t.parent = t.handle.parent().cpu().numpy()
        t.handle.close()
        t.handle = None
        self.used -= t.bytes
        t.bytes = 0
        self.evictions += 1

    def admit_all(self) -> int:
        """Make tenants resident up front, in registration order, while the
        budget allows (the resident set a serving run starts from).  Returns
        the number admitted."""
        k = 0
        for t in self.tenants.values():
            if t.handle is None and self.used + self._estimate(t) <= self.budget and self._admit(t):
                k += 1
        torch.cuda.synchronize()
        return k

    def close(self) -> None:
        """Release every tenant's handle and streams."""
        for t in self.tenants.values():
            if t.handle is not None:
                t.handle.close()
                t.handle = None
            for o in t.own:
                o.close()
            t.own.clear()
            t.stream = t.fast = None

    def state(self, tid: int):
        """(edges, parent) of a tenant on the host."""
        t = self.tenants[tid]
        if t.handle is None:
            return t.edges, t.parent
        with torch.cuda.stream(t.stream):
            return t.handle.export_edges().cpu().numpy(), t.handle.parent().cpu().numpy()

    # -- running ------------------------------------------------------------
    def _take(self, t: Tenant, now: float):
        """Head requests of a tenant that have arrived, coalesced by op."""
        q = t.queue
        if not q or q[0].t_arrive > now:
            return None
        reqs = [q.popleft()]
        if self.coalesce:
            size = len(reqs[0].batch)
            while q and q[0].t_arrive <= now and q[0].op == reqs[0].op and size + len(q[0].batch) <= self.max_coalesce:
                size += len(q[0].batch)
                reqs.append(q.popleft())
        return reqs

    def _launch(self, t: Tenant, reqs: list[Request]) -> None:
        """Apply a tenant's (coalesced) requests on its stream: a big batch
        on the tenant's high-priority stream (ordered after the tenant's
        earlier work, which has completed: one batch in flight per tenant)."""
        batch = reqs[0].batch if len(reqs) == 1 else np.concatenate([r.batch for r in reqs])
        big = self.priority_big and len(batch) >= self.big_batch
        s = t.fast if big else t.stream
        before = torch.cuda.memory_allocated()
        t.handle._stream = s
        t.handle.apply_host(reqs[0].op, batch)
        # storage the handle grew for this batch is charged to the tenant
        grown = torch.cuda.memory_allocated() - before
        t.bytes += grown
        self.used += grown
        t.event = torch.cuda.Event()
        t.event.record(s)
        t.inflight = reqs
        t.log.append((reqs[0].op, batch))

    def run(self, requests: list[Request], poll_sleep: float = 0.0) -> list[Done]:
        """Serve a trace (arrival times in seconds from now); returns the
        completion record of every request.  Python's cyclic garbage
        collector is paused while serving (a collection of a large heap would
        stall the loop and every batch in flight with it)."""
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, poll_sleep)
        finally:
            if gc_was:
                gc.enable()

    def _run(self, requests: list[Request], poll_sleep: float) -> list[Done]:
        pending = sorted(requests, key=lambda r: (r.t_arrive, r.rid))
        for t in self.tenants.values():
            t.queue.clear()
        done: list[Done] = []
        inflight: list[Tenant] = []
        t0 = time.perf_counter()
        i = 0
        total = len(pending)
        while len(done) < total:
            now = time.perf_counter() - t0
            while i < total and pending[i].t_arrive <= now:
                self.tenants[pending[i].tenant].queue.append(pending[i])
                i += 1
            # completions
            for t in list(inflight):
                if t.event.query():
                    t.handle.sync()
                    tdone = time.perf_counter() - t0
                    for r in t.inflight:
                        done.append(Done(r.rid, r.tenant, r.t_arrive, tdone, len(r.batch)))
                    t.inflight = None
                    t.last_used = tdone
                    inflight.remove(t)
            # admissions: a big batch runs alone (it waits for the small
            # batches in flight to drain, and blocks admissions while it
            # runs); small batches share the device, earliest-arrived first
            big_running = self.exclusive_big and any(len(u.log[-1][1]) >= self.big_batch for u in inflight)
            if len(inflight) < self.slots and not big_running:
                ready = [t for t in self.tenants.values() if t.inflight is None and t.queue and t.queue[0].t_arrive <= now]
                big = [t for t in ready if len(t.queue[0].batch) >= self.big_batch] if self.exclusive_big else []
                if big:
                    t = min(big, key=lambda u: u.queue[0].t_arrive)
                    if not inflight and self._admit(t):
                        self._launch(t, self._take(t, now))
                        inflight.append(t)
                else:
                    ready.sort(key=lambda t: t.queue[0].t_arrive)
                    for t in ready:
                        if len(inflight) >= self.slots:
                            break
                        if not self._admit(t):
                            continue
                        self._launch(t, self._take(t, now))
                        inflight.append(t)
            if not inflight:
                now = time.perf_counter() - t0
                ready = any(t.queue and t.queue[0].t_arrive <= now for t in self.tenants.values())
                if ready:
                    stuck = [t for t in self.tenants.values() if t.queue and t.handle is None]
                    if stuck and all(self._estimate(t) > self.budget for t in stuck):
                        raise MemoryError("a tenant does not fit the device-memory budget")
                elif i < total:
                    wait = pending[i].t_arrive - now
                    if wait > 0:
                        time.sleep(wait)
            elif poll_sleep:
                time.sleep(poll_sleep)
        return done


def run_synchronous(tenants: dict[int, tuple[int, np.ndarray, np.ndarray]], requests: list[Request],
                    flags: int = DETERMINISTIC) -> tuple[list[Done], dict[int, DynamicForest]]:
    """The plain alternative: one batch at a time in arrival order, each
    applied and synchronised before the next starts."""
    handles = {tid: DynamicForest(n, torch.from_numpy(e).cuda(), torch.from_numpy(p).cuda(), flags=flags)
               for tid, (n, e, p) in tenants.items()}
    torch.cuda.synchronize()
    done = []
    gc_was = gc.isenabled()
    gc.disable()   # as in Server.run: no collector pauses inside the timed loop
    try:
        t0 = time.perf_counter()
        for r in sorted(requests, key=lambda r: (r.t_arrive, r.rid)):
            wait = r.t_arrive - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            h = handles[r.tenant]
            h.apply_host(r.op, r.batch)
            h.sync()
            done.append(Done(r.rid, r.tenant, r.t_arrive, time.perf_counter() - t0, len(r.batch)))
    finally:
        if gc_was:
            gc.enable()
    return done, handles


def summarize(done: list[Done]) -> dict:
    lat = np.array([d.t_done - d.t_arrive for d in done]) * 1e3
    span = max(d.t_done for d in done) - min(d.t_arrive for d in done)
    upd = sum(d.updates for d in done)
    return {"updates_per_s": round(upd / span, 1), "requests": len(done), "updates": int(upd),
            "makespan_s": round(span, 4), "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                                        "p99": round(float(np.percentile(lat, 99)), 3),
                                                        "mean": round(float(lat.mean()), 3)}}
