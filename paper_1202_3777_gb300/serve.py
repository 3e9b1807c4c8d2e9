"""Continuous-batching server over several resident junction trees.

Queries (a tree and its evidence) arrive over time.  Each tree is loaded
once and keeps its potentials on the device; it owns one CUDA stream and a
number of evidence-case slots.  Whenever a tree's previous batch has
finished, the queries waiting for that tree are admitted into its next batch
as far as its slots and the device-memory budget allow: the budget covers
every tree's resident tables plus the per-case state (messages, evidence,
results) of the batches in flight, so a batch that would exceed it waits
until another batch finishes and releases its share.  Its evidence is copied
into the slots and one propagation covers the batch, so queries that arrive
while other work is on the GPU join the next batch.

Batches of different trees overlap on the device: each propagation is one
persistent kernel that claims one SM per CTA, so a batch launched while other
trees have work in flight or waiting holds at most half of the SMs
(jt_propagate_ctas), and two trees' batches run side by side on disjoint SMs;
a batch launched while the rest of the server is idle takes every SM.  Per
batch the server records the kernel's span on the GPU's global timer
(jt_get_kernel_span), from which the overlap of different trees' batches is
measured, and per query its arrival and completion times, from which p50/p99
latency follow.

This module only schedules: every step of a propagation runs in libjt's
kernels (jt_set_evidence_dense, jt_propagate_ctas, jt_get_marginals,
jt_get_log_evidence, jt_get_status).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import jt as _jt


def batch_size_class(n: int) -> int:
    """Slots a batch of n queries occupies: 1, or n rounded up to a multiple
    of 8 (the library propagates cases in blocks of 8 or 32, so the padding
    adds little work and keeps the number of recorded propagation shapes
    small)."""
    if n <= 1:
        return 1
    return (n + 7) // 8 * 8


def slots_within_budget(budget_bytes: int, table_bytes: int, case_bytes: int, max_batch: int) -> int:
    """Evidence-case slots a tree may keep when its tables take table_bytes of
    budget_bytes and every slot takes case_bytes (0 if even one slot does not
    fit)."""
    room = budget_bytes - table_bytes
    if room < case_bytes:
        return 0
    n = min(max_batch, room // max(1, case_bytes))
    if n >= 8:
        n = n // 8 * 8
    return int(n)


def admissible(waiting: int, slots: int, free_bytes: int, case_bytes: int) -> int:
    """Queries a tree may admit into its next batch: no more than are
    waiting or than its slots hold, and only as many as the device-memory
    budget left by the batches in flight can carry (the batch reserves the
    slots it occupies, rounded to its size class)."""
    n = min(waiting, slots)
    while n > 0 and batch_size_class(n) * case_bytes > free_bytes:
        n = n - 1 if n <= 8 else (n - 1) // 8 * 8
    return max(n, 0)


def sm_share(n_sm: int, others_busy: bool) -> int:
    """CTAs a batch's propagation may hold: half of the SMs when other trees
    have work in flight or waiting (so two trees' batches run side by side),
    every SM (0) otherwise."""
    return max(1, n_sm // 2) if others_busy else 0


def overlapping_pairs(spans) -> int:
    """Pairs of kernel spans (tree, start, end) of different trees that
    overlap in time on the GPU."""
    n = 0
    for i in range(len(spans)):
        for j in range(i + 1, len(spans)):
            a, b = spans[i], spans[j]
            if a[0] != b[0] and a[1] < b[2] and b[1] < a[2]:
                n += 1
    return n


@dataclass
class Query:
    qid: int
    tree: str
    states: np.ndarray               # int16 [n_vars], -1 = unobserved
    arrival: float = 0.0
    done: float = 0.0
    marginals: Optional[np.ndarray] = None
    log_z: float = float("nan")
    status: int = -1
    batch: int = 0                   # queries in the batch that served it


@dataclass
class _Resident:
    name: str
    handle: object
    n_vars: int
    slots: int
    stream: object
    work: int                        # clique entries per case (Eq. 4 numerator)
    case_bytes: int = 0              # device bytes of one case slot
    table_bytes: int = 0             # device bytes of everything else of the tree
    queue: collections.deque = field(default_factory=collections.deque)
    batch: List[Query] = field(default_factory=list)
    event: object = None
    reserved: int = 0                # budget bytes held by the batch in flight


class Server:
    """Keeps trees resident and serves queries with continuous batching.

    trees: name -> synth.Tree (or any object with card, cliques, parent,
    pot); budget_bytes bounds the device memory of the trees' tables and of
    the batches in flight; max_batch bounds the slots of one tree."""

    def __init__(self, trees: Dict[str, object], budget_bytes: int = 60 << 30, max_batch: int = 64,
                 compute: int = _jt.JT_F32):
        import torch
        self._torch = torch
        self.trees: Dict[str, _Resident] = {}
        self.budget = int(budget_bytes)
        self.n_sm = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
        used = 0
        for name, tree in trees.items():
            h = _jt.jt_load_synth(tree, compute=compute, max_cases=max_batch)
            info = h.info
            table_bytes = int(info.device_bytes - max_batch * info.case_bytes)
            if used + info.device_bytes > budget_bytes:
                # keep as many slots as the budget left by the other trees' tables allows
                slots = slots_within_budget(budget_bytes - used, table_bytes, int(info.case_bytes), max_batch)
                h.free()
                if slots == 0:
                    raise MemoryError(f"tree {name} does not fit in the remaining device-memory budget")
                h = _jt.jt_load_synth(tree, compute=compute, max_cases=slots)
            slots = int(h.info.max_cases)
            used += table_bytes
            self.trees[name] = _Resident(name, h, int(h.info.n_vars), slots, torch.cuda.Stream(),
                                         int(h.info.work_per_case), int(h.info.case_bytes), table_bytes)
        self.table_bytes = used
        self.completed: List[Query] = []
        self.spans: List[tuple] = []        # (tree, kernel start ns, kernel end ns, queries)
        self.deferred = 0                   # launches the memory budget held back

    @property
    def free_bytes(self) -> int:
        return self.budget - self.table_bytes - sum(r.reserved for r in self.trees.values())

    def warm_up(self):
        """Record every batch shape once, on all SMs and on half of them
        (propagation graphs are built on first use)."""
        for r in self.trees.values():
            sizes = sorted({batch_size_class(n) for n in range(1, r.slots + 1)})
            for n in sizes:
                _jt.jt_set_evidence_dense(r.handle, 0, np.full((n, r.n_vars), -1, np.int16), stream=r.stream)
                for cap in {0, sm_share(self.n_sm, True)}:
                    _jt.jt_propagate_ctas(r.handle, 0, n, cap, r.stream)
            r.stream.synchronize()

    def submit(self, q: Query, now: Optional[float] = None):
        q.arrival = time.perf_counter() if now is None else now
        self.trees[q.tree].queue.append(q)

    def _finish(self, r: _Resident):
        n = len(r.batch)
        m = _jt.jt_get_marginals(r.handle, 0, n, stream=r.stream)
        lz = _jt.jt_get_log_evidence(r.handle, 0, n, stream=r.stream)
        st = _jt.jt_get_status(r.handle, 0, n)
        t0, t1 = _jt.jt_get_kernel_span(r.handle)
        self.spans.append((r.name, t0, t1, n))
        t = time.perf_counter()
        for i, q in enumerate(r.batch):
            q.marginals, q.log_z, q.status, q.done, q.batch = m[i], float(lz[i]), int(st[i]), t, n
            self.completed.append(q)
        r.batch, r.event, r.reserved = [], None, 0

    def _plan(self, r: _Resident):
        """(queries to admit, CTA limit) for the tree's next batch."""
        take = admissible(len(r.queue), r.slots, self.free_bytes, r.case_bytes)
        others = any(o is not r and (o.event is not None or o.queue) for o in self.trees.values())
        return take, sm_share(self.n_sm, others)

    def _issue(self, r: _Resident, batch: List[Query], n: int, cap: int):
        ev = np.full((n, r.n_vars), -1, np.int16)
        for i, q in enumerate(batch):
            ev[i] = q.states
        _jt.jt_set_evidence_dense(r.handle, 0, ev, stream=r.stream)
        _jt.jt_propagate_ctas(r.handle, 0, n, cap, r.stream)
        r.event = self._torch.cuda.Event()
        r.event.record(r.stream)

    def _launch(self, r: _Resident) -> bool:
        take, cap = self._plan(r)
        if take == 0:
            self.deferred += 1
            return False
        batch = [r.queue.popleft() for _ in range(take)]
        n = batch_size_class(take)
        r.batch = batch
        r.reserved = n * r.case_bytes
        self._issue(r, batch, n, cap)
        return True

    def poll(self) -> int:
        """Finish completed batches and start the next batch of every idle
        tree with waiting queries; returns the number of batches in flight."""
        busy = 0
        for r in self.trees.values():
            if r.event is not None and r.event.query():
                self._finish(r)
        for r in self.trees.values():
            if r.event is None and r.queue:
                self._launch(r)
            busy += r.event is not None
        return busy

    def drain(self):
        while self.poll() or any(r.queue for r in self.trees.values()):
            pass

    def run_arrivals(self, arrivals: List[tuple]):
        """Serve (offset_seconds, Query) arrivals in real time: each query is
        submitted once its offset has passed; returns the completed queries."""
        arrivals = sorted(arrivals, key=lambda a: a[0])
        t0 = time.perf_counter()
        i = 0
        while True:
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                self.submit(arrivals[i][1], t0 + arrivals[i][0])
                i += 1
            # batches start and finish while later queries are still to arrive
            busy = self.poll()
            if i >= len(arrivals) and busy == 0 and not any(r.queue for r in self.trees.values()):
                break
        return self.completed

    def free(self):
        for r in self.trees.values():
            r.handle.free()
        self.trees = {}


def latency_summary(queries: List[Query], work: Dict[str, int]) -> dict:
    """p50/p99 latency (ms), throughput in clique entries per second."""
    lat = np.array([q.done - q.arrival for q in queries]) * 1e3
    span = max(q.done for q in queries) - min(q.arrival for q in queries)
    entries = sum(work[q.tree] for q in queries)
    return {"queries": len(queries), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "clique_entries_per_s": entries / span if span > 0 else float("nan"), "span_s": span}
