"""Continuous-batching request loop for CSPH-TVD simulations on one GPU.

Requests (a grid and its physical parameters, a number of steps) arrive over
time.  The server keeps every admitted request's state resident on the
device in its own solver handle, admits waiting requests as soon as their
device footprint (``cspht_device_bytes``) fits the memory budget and a slot
is free, and advances all active requests together: each scheduler tick
enqueues a chunk of steps for every active request on that request's own
CUDA stream (each chunk is a replay of the handle's step graph), so the
kernels of different requests overlap on the GPU.  A request retires when
its steps are done; its handle is destroyed and its memory admits the next
request.  Time-to-solution is completion minus arrival.

The scheduler is host code; every step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
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


class _Active:
    def __init__(self, req, w, sim, stream, now):
        import torch
        self.req, self.w, self.sim, self.stream = req, w, sim, stream
        self.steps_left = req["steps"]
        self.admitted = now
        self.event = torch.cuda.Event()
        self.inflight = False


class Server:
    """Admits requests against ``budget_bytes`` of device memory and at most
    ``max_active`` at a time; ``chunk`` steps are enqueued per tick."""

    def __init__(self, budget_bytes: int, max_active: int = 32, chunk: int = 10, precision: int = 32,
                 keep_state: bool = False):
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.chunk = chunk
        self.precision = precision
        self.keep_state = keep_state
        self.used = 0
        self.waiting: deque = deque()
        self.active: list[_Active] = []
        self.results: list[Result] = []
        self.max_used = 0

    def footprint(self, req) -> int:
        e = req["edge"]
        return cspht.device_bytes((e, e, e), self.precision, cspht.PATH_FAST)

    def submit(self, req):
        if self.footprint(req) > self.budget:
            raise ValueError(f"request {req['id']} needs more than the whole budget")
        self.waiting.append(req)

    def _admit(self, now):
        import torch
        while self.waiting and len(self.active) < self.max_active:
            req = self.waiting[0]
            need = self.footprint(req)
            if self.used + need > self.budget:
                break
            self.waiting.popleft()
            w = wl.request_workload(req)
            stream = torch.cuda.Stream()
            sim = cspht.Sim.from_workload(w, precision=self.precision, path=cspht.PATH_FAST)
            sim.set_stream(stream)
            sim.set_primitive(np.ascontiguousarray(w.W))
            self.used += need
            self.max_used = max(self.max_used, self.used)
            self.active.append(_Active(req, w, sim, stream, now))

    def _tick(self, now):
        """Enqueue the next chunk for every idle request; retire finished ones."""
        still = []
        for a in self.active:
            if a.inflight and not a.event.query():
                still.append(a)
                continue
            a.inflight = False
            if a.steps_left == 0:
                a.sim.sync()
                tot = a.sim.totals()
                st = a.sim.get_state() if self.keep_state else None
                done = time.perf_counter()
                self.results.append(Result(a.req["id"], a.w.cells, a.req["steps"], a.req["arrival_abs"],
                                           a.admitted, done, tot, st))
                a.sim.close()
                self.used -= self.footprint(a.req)
                continue
            n = min(self.chunk, a.steps_left)
            a.sim.advance(n, a.w.cfl)
            a.event.record(a.stream)
            a.steps_left -= n
            a.inflight = True
            still.append(a)
        self.active = still

    def run(self, requests, realtime: bool = True):
        """Replays ``requests`` (dicts with an ``arrival`` time in seconds) and
        serves them to completion.  Returns the list of results."""
        pending = deque(sorted(requests, key=lambda r: r["arrival"]))
        t0 = time.perf_counter()
        while pending or self.waiting or self.active:
            now = time.perf_counter()
            while pending and (not realtime or pending[0]["arrival"] <= now - t0):
                r = dict(pending.popleft())
                r["arrival_abs"] = t0 + r["arrival"] if realtime else now
                self.submit(r)
            self._admit(now)
            self._tick(now)
            if not self.active and not self.waiting and pending and realtime:
                time.sleep(max(0.0, min(0.002, pending[0]["arrival"] - (time.perf_counter() - t0))))
        self.makespan = time.perf_counter() - t0
        return self.results

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
        }


def run_alone(req, precision=32):
    """One request on its own (reference for the in-the-mix results)."""
    w = wl.request_workload(req)
    with cspht.Sim.from_workload(w, precision=precision, path=cspht.PATH_FAST) as s:
        s.set_primitive(np.ascontiguousarray(w.W))
        s.advance(req["steps"], w.cfl)
        s.sync()
        return s.totals(), s.get_state()
