"""Continuous-batching request loop for CSPH-TVD simulations on one GPU.

Requests (a grid and its physical parameters, a number of steps) arrive over
time.  The server keeps every admitted request's state resident on the
device in its own solver handle, admits waiting requests as soon as their
device footprint (``cspht_device_bytes``) fits the memory budget and a slot
is free, and advances all active requests together.  A request retires when
its steps are done; its handle is destroyed and its memory admits the next
request.  Time-to-solution is completion minus arrival.

Per-request mode (the default) enqueues every request's chunk of steps on
its own stream, so requests progress independently and their kernels
overlap on the GPU; smaller requests get higher-priority streams (turn off
with ``priorities=False``), so the block scheduler serves their kernels first
instead of queueing them behind the largest requests'.  Batched mode
(``batched=True``): all active requests advance in lockstep, each with its
own dt, through a ``cspht.Batch`` of the active set: one launch of each step
kernel for all of them, the fused stages as persistent kernels that take
(request, tile, z chunk) items from a device counter, two steps at a time
replayed from the batch's CUDA graph.  The batch is rebuilt when the set of
active requests changes.  (Requests whose boundaries the batch cannot take
run through ``cspht_batch_step``, a captured graph of every request's own
step kernels.)  Lockstep makes every tick last as long as the largest
request's steps, so small requests wait for it.  Adaptive mode
(``adaptive=True``) takes the lockstep batch while requests wait for
admission (the GPU is saturated and one launch per step kernel serves more
cells per second) and per-request streams while none wait (a new request
starts at once on its own stream instead of waiting for the batch's tick).

A request's payload (its initial state and potential) stands for the data
a client sends with it: ``run`` takes the payloads already built, or builds
each one from the request's parameters when the request is admitted.

With per-request streams, set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) to at
least ``max_active`` before CUDA starts in the process: with the driver's
default of 8 hardware queues, a request's setup and result kernels wait
behind the work of other streams that share its queue.

The scheduler is host code; every step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import itertools
import time
from collections import deque

import numpy as np

from . import cspht
from . import workloads as wl


@dataclasses.dataclass
class Result:
    id: int
    cells: int
    steps: int
    arrival: float
    admitted: float
    done: float
    totals: np.ndarray
    state: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


_uid = itertools.count()


class _Active:
    def __init__(self, req, w, sim, stream, now):
        import torch
        self.uid = next(_uid)
        self.req, self.w, self.sim, self.stream = req, w, sim, stream
        self.steps_left = req["steps"]
        self.admitted = now
        self.pending = deque()  # events of the chunks enqueued on the request's stream, oldest first

    def busy(self) -> bool:
        """Drops the finished chunks; True while one is still in flight."""
        while self.pending and self.pending[0].query():
            self.pending.popleft()
        return bool(self.pending)


class Server:
    """Admits requests against ``budget_bytes`` of device memory and at most
    ``max_active`` at a time; ``chunk`` steps per request per tick, up to
    ``ahead`` chunks enqueued per request with per-request streams."""

    def __init__(self, budget_bytes: int, max_active: int = 32, chunk: int = 10, precision: int = 32,
                 keep_state: bool = False, batched: bool = False, cfl: float = 0.4,
                 priorities: bool = True, adaptive: bool = False, ahead: int = 2):
        import torch
        self.ahead = max(1, int(ahead))  # chunks in flight per request (per-request streams)
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.chunk = chunk
        self.precision = precision
        self.keep_state = keep_state
        self.adaptive = adaptive
        self.batched = batched and not adaptive
        self.cfl = cfl
        # stream priorities by size (per-request mode): smaller requests get
        # higher-priority streams, so the block scheduler serves their kernels
        # first and they do not wait behind the largest ones
        self.priorities = priorities and not self.batched
        self.prio_range = torch.cuda.Stream.priority_range() if self.priorities else (0, 0)
        self.used = 0
        self.waiting: deque = deque()
        self.active: list[_Active] = []
        self.results: list[Result] = []
        self.max_used = 0
        self.stream = torch.cuda.Stream()
        self.result_stream = torch.cuda.Stream(priority=torch.cuda.Stream.priority_range()[1])
        self.batch_event = torch.cuda.Event()
        self.batch_inflight = False
        self.graph = None
        self.graph_key = None
        self.graph_launches = 0
        self.max_waiting = 0  # longest queue of arrived, not yet admitted requests
        self.multi = None      # cspht.Batch of the active set (batched mode)
        self.multi_key = None
        self.multi_ticks = 0   # ticks that ran through a cspht.Batch
        self.stream_ticks = 0  # ticks that enqueued per-request chunks
        self.payloads = None   # request id -> Workload built before the replay (run())

    def footprint(self, req) -> int:
        e = req["edge"]
        return cspht.device_bytes((e, e, e), self.precision, cspht.PATH_FAST)

    def submit(self, req):
        if self.footprint(req) > self.budget:
            raise ValueError(f"request {req['id']} needs more than the whole budget")
        self.waiting.append(req)

    def _priority(self, cells: int) -> int:
        """Stream priority: the greatest for grids up to 64^3, the middle up to
        128^3, the least above (CUDA: lower numbers are higher priorities)."""
        least, greatest = self.prio_range
        if not self.priorities or least == greatest:
            return 0
        if cells <= 64 ** 3:
            return greatest
        if cells <= 128 ** 3:
            return (least + greatest) // 2
        return least

    def _admit(self, now):
        import torch
        while self.waiting and len(self.active) < self.max_active:
            req = self.waiting[0]
            need = self.footprint(req)
            if self.used + need > self.budget:
                break
            self.waiting.popleft()
            w = self.payloads.get(req["id"]) if self.payloads else None
            w = w if w is not None else wl.request_workload(req)
            stream = torch.cuda.Stream(priority=self._priority(w.cells))
            sim = cspht.Sim.from_workload(w, precision=self.precision, path=cspht.PATH_FAST)
            sim.set_stream(stream)
            sim.set_primitive(np.ascontiguousarray(w.W))
            a = _Active(req, w, sim, stream, now)
            self.used += need
            self.max_used = max(self.max_used, self.used)
            self.active.append(a)

    def _retire(self, a):
        a.sim.sync()
        # the result's reductions on a greatest-priority stream, so that they do
        # not queue behind the other requests' kernels while the host waits
        a.sim.set_stream(self.result_stream)
        tot = a.sim.totals()
        st = a.sim.get_state() if self.keep_state else None
        done = time.perf_counter()
        self.results.append(Result(a.req["id"], a.w.cells, a.req["steps"], a.req["arrival_abs"],
                                   a.admitted, done, tot, st))
        a.sim.close()
        self.used -= self.footprint(a.req)

    def _tick_batched(self):
        """Retire finished requests, then advance all others together by up to
        ``chunk`` steps: one launch of each step kernel for all of them
        (cspht_batch_*: persistent fused kernels over every member's tiles,
        two steps at a time replayed from the batch's own CUDA graph).  A
        member whose boundaries the batch cannot take runs the active set
        through the per-handle batch graph instead."""
        import torch
        if self.batch_inflight and not self.batch_event.query():
            return
        self.batch_inflight = False
        if any(a.steps_left == 0 for a in self.active) and self.multi is not None:
            self.multi.close()  # before its members are freed
            self.multi, self.multi_key = None, None
        still = []
        for a in self.active:
            if a.steps_left == 0:
                self._retire(a)
            else:
                still.append(a)
        self.active = still
        if not self.active:
            return
        sims = [a.sim for a in self.active]
        n = min(self.chunk, min(a.steps_left for a in self.active))
        key = tuple(a.uid for a in self.active)
        if self.multi_key != key:
            if self.multi is not None:
                self.multi.close()
            self.multi, self.multi_key = None, key
            try:
                self.multi = cspht.Batch(sims)
            except cspht.CsphtError as e:
                if e.code != cspht.EINVAL:
                    raise
        if self.multi is not None:
            self.multi.advance(n, self.cfl, self.stream)
            self.graph_launches += 1
            self.multi_ticks += 1
            for a in self.active:
                a.steps_left -= n
            self.batch_event.record(self.stream)
            self.batch_inflight = True
            return
        pairs, single = n // 2, n % 2
        if pairs:
            key = tuple(a.uid for a in self.active)
            if self.graph is None or self.graph_key != key:
                # captured again whenever the members change (a retired member's
                # handle is freed, so an old graph is never replayed)
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.stream(self.stream):
                    self.graph.capture_begin(capture_error_mode="thread_local")
                    try:
                        for _ in range(2):
                            cspht.batch_step(sims, self.cfl, self.stream)
                    finally:
                        self.graph.capture_end()
                self.graph_key = key
            with torch.cuda.stream(self.stream):
                for _ in range(pairs):
                    self.graph.replay()
                    self.graph_launches += 1
        if single:  # an odd step flips every member's buffers: the graph no longer fits them
            cspht.batch_step(sims, self.cfl, self.stream)
            self.graph, self.graph_key = None, None
        for a in self.active:
            a.steps_left -= n
        self.batch_event.record(self.stream)
        self.batch_inflight = True

    def _tick_adaptive(self, now):
        """Lockstep batch while requests wait for admission, per-request
        streams otherwise.  A switch waits until the other mode's work is
        done: every request's own stream before a batch tick, the batch
        before a streams tick."""
        if self.waiting:
            if any(a.busy() for a in self.active):
                return
            self._tick_batched()
        else:
            if self.batch_inflight and not self.batch_event.query():
                return
            self.batch_inflight = False
            if self.multi is not None:  # a member may retire in streams mode; the batch must not outlive it
                self.multi.close()
                self.multi, self.multi_key = None, None
            self.graph, self.graph_key = None, None
            self._tick(now)

    def _tick(self, now):
        """Keep ``ahead`` chunks enqueued on every request's stream (so that its
        GPU work does not run out while the host admits or retires others);
        retire finished requests."""
        import torch
        self.stream_ticks += 1
        still = []
        for a in self.active:
            busy = a.busy()
            if a.steps_left == 0 and not busy:
                self._retire(a)
                continue
            while a.steps_left > 0 and len(a.pending) < self.ahead:
                n = min(self.chunk, a.steps_left)
                a.sim.advance(n, a.w.cfl)
                ev = torch.cuda.Event()
                ev.record(a.stream)
                a.pending.append(ev)
                a.steps_left -= n
            still.append(a)
        self.active = still

    def run(self, requests, realtime: bool = True, payloads: dict | None = None):
        """Replays ``requests`` (dicts with an ``arrival`` time in seconds) and
        serves them to completion.  ``payloads`` maps a request id to its
        Workload when the payloads arrive built with the requests; a request
        without one is built from its parameters at admission.  Returns the
        list of results."""
        self.payloads = payloads
        pending = deque(sorted(requests, key=lambda r: r["arrival"]))
        # offered load: the cell-updates the stream asks for over its arrival span
        span = max(r["arrival"] for r in requests) if requests else 0.0
        work = sum(r["edge"] ** 3 * r["steps"] for r in requests)
        self.offered = work / span / 1e9 if span > 0 else None
        t0 = time.perf_counter()
        while pending or self.waiting or self.active:
            now = time.perf_counter()
            while pending and (not realtime or pending[0]["arrival"] <= now - t0):
                r = dict(pending.popleft())
                r["arrival_abs"] = t0 + r["arrival"] if realtime else now
                self.submit(r)
            self._admit(now)
            self.max_waiting = max(self.max_waiting, len(self.waiting))
            if self.adaptive:
                self._tick_adaptive(now)
            elif self.batched:
                self._tick_batched()
            else:
                self._tick(now)
            if not self.active and not self.waiting and pending and realtime:
                time.sleep(max(0.0, min(0.002, pending[0]["arrival"] - (time.perf_counter() - t0))))
        self.makespan = time.perf_counter() - t0
        return self.results

    def mode(self) -> str:
        if self.adaptive:
            return "adaptive: one launch per step kernel while requests wait, else per-request streams"
        if self.batched:
            return "one launch per step kernel" if self.multi_ticks else "batched graph"
        return "per-request streams, priorities by size" if self.priorities else "per-request streams"

    def metrics(self) -> dict:
        lat = np.array([r.latency for r in self.results])
        cells = sum(r.cells * r.steps for r in self.results)
        return {
            "requests": len(self.results),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "aggregate_gcell_s": cells / self.makespan / 1e9,
            "makespan_s": self.makespan,
            "cell_updates": cells,
            "peak_device_bytes": self.max_used,
            "budget_bytes": self.budget,
            "mode": self.mode(),
            "batch_ticks": self.multi_ticks,
            "batch_graph_launches": self.graph_launches,
            "max_waiting": self.max_waiting,
            "offered_gcell_s": self.offered,
        }


def pinned(w):
    """The payload w with its state and potential in page-locked host memory,
    as a client's transfer buffers would be: the uploads at admission then run
    at the bus's rate instead of through the driver's staging copies.  Falls
    back to w itself when page-locked memory cannot be had."""
    import torch
    try:
        Wt = torch.from_numpy(np.ascontiguousarray(w.W)).pin_memory()
        Pt = torch.from_numpy(np.ascontiguousarray(w.psi)).pin_memory()
    except RuntimeError:
        return w
    p = dataclasses.replace(w, W=Wt.numpy(), psi=Pt.numpy())
    p.pinned_buffers = (Wt, Pt)  # keep the page-locked memory alive with the payload
    return p


def run_alone(req, precision=32):
    """One request on its own (reference for the in-the-mix results)."""
    w = wl.request_workload(req)
    with cspht.Sim.from_workload(w, precision=precision, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(req["steps"], w.cfl)
        s.sync()
        return s.totals(), s.get_state()
