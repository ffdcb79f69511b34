"""Continuous-batching request loop over the batched C ABI.

Simulations arrive over time (seeded Poisson process).  The library makes the device-side
decisions: ``apic_batch_admit`` lets a simulation join the resident batch only while the
device footprints of the admitted members (their ``apic_workspace_size``) stay under the
memory budget (else ``APIC_ERR_OOM`` and nothing changes), and ``apic_batch_run`` advances
every member to the nearest completion (at most a few batched steps) and takes the finished
ones out of the batch.  This module is the thin host driver around those two calls: it keeps
the arrival clock and the FIFO queue (the head is admitted first and nothing overtakes it),
rejects at arrival a request whose footprint can never fit the budget, evicts a request whose
admission or read-back fails and keeps serving the others, and records completion latency =
finish time - arrival time.

:class:`Scheduler` takes the GPU work as callables, so the loop itself runs without a device.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    steps: int
    footprint: int          # device bytes while resident
    particles: int
    payload: object = None  # whatever the launcher needs to build the simulation
    admitted: float = -1.0
    finished: float = -1.0


@dataclass
class Report:
    completed: int
    particle_steps: float
    makespan: float
    latencies: list = field(default_factory=list)
    max_resident: int = 0
    max_bytes: int = 0
    batched_steps: int = 0
    rejected: list = field(default_factory=list)   # request ids that can never fit the budget
    failed: list = field(default_factory=list)     # (request id, reason) evicted after an error

    @property
    def throughput(self) -> float:
        return self.particle_steps / self.makespan if self.makespan > 0 else 0.0

    def percentile(self, q: float) -> float:
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


class Deferred(Exception):
    """admit() raises this when the request does not fit the budget now (APIC_ERR_OOM)."""


class Scheduler:
    """FIFO admission without overtaking, rejection of requests that can never fit,
    eviction on errors, latency bookkeeping.

    admit(req) -> handle    build + upload the simulation and admit it (apic_batch_admit);
                            raises Deferred when it does not fit now, any other exception
                            when it fails (the request is then evicted)
    run(n) -> (handles, k)  at most n batched steps, to the nearest completion
                            (apic_batch_run); returns the finished members and the steps k
    retire(req, handle)     read the result back and free the simulation; an exception
                            marks the request failed
    resident_bytes()        device bytes of the admitted members
    now()                   seconds since start
    """

    def __init__(self, budget_bytes: int, max_resident: int, admit, run, retire, now, resident_bytes,
                 max_chunk: int = 8, idle_wait=None):
        self.budget = budget_bytes
        self.max_resident = max_resident
        self._admit, self._run, self._retire, self._now = admit, run, retire, now
        self._resident_bytes = resident_bytes
        self.max_chunk = max_chunk
        self.idle_wait = idle_wait or (lambda dt: time.sleep(max(0.0, min(dt, 0.01))))

    def run(self, requests: list[Request]) -> Report:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque[Request] = collections.deque()
        resident: dict[object, Request] = {}
        rep = Report(0, 0.0, 0.0)
        t_first = None
        while pending or queue or resident:
            now = self._now()
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if r.footprint > self.budget:          # can never be admitted
                    rep.rejected.append(r.rid)
                else:
                    queue.append(r)
            # admit in arrival order while the head fits
            while queue and len(resident) < self.max_resident:
                r = queue[0]
                try:
                    h = self._admit(r)
                except Deferred:
                    break
                except Exception as e:                 # evict it, keep serving the rest
                    queue.popleft()
                    rep.failed.append((r.rid, f"admission: {e}"))
                    continue
                queue.popleft()
                r.admitted = self._now()
                resident[h] = r
                t_first = r.arrival if t_first is None else min(t_first, r.arrival)
            rep.max_resident = max(rep.max_resident, len(resident))
            rep.max_bytes = max(rep.max_bytes, self._resident_bytes())
            if not resident:
                if queue:
                    raise RuntimeError(f"request {queue[0].rid} fits the budget but was not admitted into an empty batch")
                if pending:
                    self.idle_wait(pending[0].arrival - now)
                continue
            done, k = self._run(self.max_chunk)
            rep.batched_steps += k
            for r in resident.values():
                rep.particle_steps += float(r.particles) * k
            for h in done:
                r = resident.pop(h)
                try:
                    self._retire(r, h)
                except Exception as e:
                    rep.failed.append((r.rid, f"read-back: {e}"))
                    continue
                r.finished = self._now()
                rep.completed += 1
                rep.latencies.append(r.finished - r.arrival)
        rep.makespan = self._now() - (t_first or 0.0)
        return rep


def poisson_arrivals(rng: np.random.Generator, rate: float, count: int) -> np.ndarray:
    """Arrival times of `count` requests of a Poisson process with the given rate (1/s)."""
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serve_gpu(requests: list[Request], make_sim, batch, budget_bytes: int, max_resident: int, max_chunk: int = 8,
              keep_state: bool = False):
    """Run the loop on the GPU.  make_sim(req) -> Sim (uploaded); batch: apic.Batch.
    Returns the report and, per request id, its final total momentum (or, with keep_state,
    its downloaded particle state)."""
    import torch

    from . import apic

    t0 = time.perf_counter()
    results = {}

    def admit(r):
        # build the simulation only when the library's ledger says it fits now (the
        # library checks again when it admits it)
        if batch.resident_bytes() + r.footprint > budget_bytes:
            raise Deferred()
        sim = make_sim(r)
        try:
            batch.admit(sim, r.steps, r.footprint, budget_bytes)
        except apic.ApicError as e:
            sim.close()
            if e.status == apic.APIC_ERR_OOM:
                raise Deferred() from e
            raise
        return sim

    def run(n):
        return batch.run(n)

    def retire(r, sim):
        try:
            results[r.rid] = sim.download() if keep_state else sim.momentum("particles")
        finally:
            sim.close()

    def now():
        return time.perf_counter() - t0

    sched = Scheduler(budget_bytes, max_resident, admit, run, retire, now, batch.resident_bytes, max_chunk=max_chunk)
    rep = sched.run(requests)
    torch.cuda.synchronize()
    return rep, results
