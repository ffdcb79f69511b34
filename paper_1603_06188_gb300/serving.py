"""Continuous-batching request loop over the batched C ABI (``apic_batch_*``).

Simulations arrive over time (seeded Poisson process).  A request is admitted, in arrival
order, as soon as its device footprint (its workspace, from ``apic_workspace_size``) fits
under the memory budget and a member slot is free; its particles are uploaded and it joins
the resident batch between two batched steps, while the others keep running.  Every loop
iteration advances all residents by a few batched steps (never past the nearest
completion); finished simulations are downloaded, leave the batch and free their memory.
Completion latency = finish time - arrival time.

The scheduling decisions (admission, step chunking, retirement) are host logic in
:class:`Scheduler`, which takes the GPU work as callables so it can be exercised without a
device.
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

    @property
    def throughput(self) -> float:
        return self.particle_steps / self.makespan if self.makespan > 0 else 0.0

    def percentile(self, q: float) -> float:
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


class Scheduler:
    """Admission by memory budget (FIFO, no overtaking), step chunking and retirement.

    admit(req) -> handle      build + upload the simulation and add it to the batch
    step(n)                   n batched steps of every resident
    retire(req, handle)       download the result, leave the batch, free memory
    now()                     seconds since start
    """

    def __init__(self, budget_bytes: int, max_resident: int, admit, step, retire, now, max_chunk: int = 8,
                 idle_wait=None):
        self.budget = budget_bytes
        self.max_resident = max_resident
        self._admit, self._step, self._retire, self._now = admit, step, retire, now
        self.max_chunk = max_chunk
        self.idle_wait = idle_wait or (lambda dt: time.sleep(max(0.0, min(dt, 0.01))))

    def run(self, requests: list[Request]) -> Report:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque[Request] = collections.deque()
        resident: dict[int, tuple[Request, object, int]] = {}
        used = 0
        rep = Report(0, 0.0, 0.0)
        t_first = None
        while pending or queue or resident:
            now = self._now()
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # admit in arrival order while the head fits
            while queue and len(resident) < self.max_resident and used + queue[0].footprint <= self.budget:
                r = queue.popleft()
                if r.footprint > self.budget:
                    raise ValueError(f"request {r.rid} can never fit the budget")
                h = self._admit(r)
                r.admitted = self._now()
                used += r.footprint
                resident[r.rid] = (r, h, r.steps)
                t_first = r.arrival if t_first is None else min(t_first, r.arrival)
            rep.max_resident = max(rep.max_resident, len(resident))
            rep.max_bytes = max(rep.max_bytes, used)
            if not resident:
                if queue:
                    raise ValueError(f"request {queue[0].rid} does not fit the budget")
                if pending:
                    self.idle_wait(pending[0].arrival - now)
                continue
            chunk = min(self.max_chunk, min(left for (_, _, left) in resident.values()))
            self._step(chunk)
            rep.batched_steps += chunk
            for rid in list(resident):
                r, h, left = resident[rid]
                left -= chunk
                rep.particle_steps += float(r.particles) * chunk
                if left == 0:
                    self._retire(r, h)
                    r.finished = self._now()
                    used -= r.footprint
                    del resident[rid]
                    rep.completed += 1
                    rep.latencies.append(r.finished - r.arrival)
                else:
                    resident[rid] = (r, h, left)
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

    t0 = time.perf_counter()
    results = {}

    def admit(r):
        sim = make_sim(r)
        batch.add(sim)
        return sim

    def step(n):
        batch.step(n)

    def retire(r, sim):
        batch.remove(sim)          # synchronises with the batch
        results[r.rid] = sim.download() if keep_state else sim.momentum("particles")
        sim.close()
        del sim

    def now():
        return time.perf_counter() - t0

    sched = Scheduler(budget_bytes, max_resident, admit, step, retire, now, max_chunk=max_chunk)
    rep = sched.run(requests)
    torch.cuda.synchronize()
    return rep, results
