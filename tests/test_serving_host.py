"""Host logic of the serving loop (no GPU): FIFO admission under a memory budget,
continuous batching (requests join while others are resident), step chunking that never
overshoots a completion, and latency bookkeeping, on a simulated clock."""
import numpy as np
import pytest

from paper_1603_06188_gb300.serving import Request, Scheduler, poisson_arrivals


class FakeGPU:
    """Each batched step costs `step_cost` seconds of simulated time; admission is free."""

    def __init__(self, step_cost=0.01):
        self.t = 0.0
        self.step_cost = step_cost
        self.resident = {}
        self.steps_done = {}
        self.log = []

    def now(self):
        return self.t

    def admit(self, r):
        self.resident[r.rid] = r
        self.steps_done[r.rid] = 0
        self.log.append(("admit", r.rid, self.t, len(self.resident)))
        return r.rid

    def step(self, n):
        for rid in self.resident:
            self.steps_done[rid] += n
        self.t += n * self.step_cost

    def retire(self, r, h):
        assert self.steps_done[r.rid] == r.steps, "a simulation must get exactly its steps"
        del self.resident[r.rid]
        self.log.append(("retire", r.rid, self.t, len(self.resident)))

    def wait(self, dt):
        self.t += max(dt, 1e-6)


def make_requests(n, seed=0, rate=50.0):
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(rng, rate, n)
    return [Request(i, float(arr[i]), int(rng.integers(5, 40)), int(rng.integers(1, 10)) * 100, int(rng.integers(1000, 5000)))
            for i in range(n)]


def test_every_request_gets_exactly_its_steps_and_latency_is_recorded():
    gpu = FakeGPU()
    reqs = make_requests(60)
    sched = Scheduler(budget_bytes=2000, max_resident=8, admit=gpu.admit, step=gpu.step, retire=gpu.retire,
                      now=gpu.now, max_chunk=4, idle_wait=gpu.wait)
    rep = sched.run(reqs)
    assert rep.completed == 60
    assert len(rep.latencies) == 60
    assert all(r.finished >= r.admitted >= r.arrival for r in reqs)
    assert rep.particle_steps == sum(r.particles * r.steps for r in reqs)
    assert rep.max_bytes <= 2000 and rep.max_resident <= 8
    assert rep.percentile(99) >= rep.percentile(50) > 0


def test_admission_is_fifo_and_continuous():
    gpu = FakeGPU()
    reqs = make_requests(40, seed=1, rate=200.0)
    sched = Scheduler(budget_bytes=1500, max_resident=6, admit=gpu.admit, step=gpu.step, retire=gpu.retire,
                      now=gpu.now, idle_wait=gpu.wait)
    sched.run(reqs)
    admits = [e for e in gpu.log if e[0] == "admit"]
    assert [e[1] for e in admits] == sorted(e[1] for e in admits)      # arrival order kept
    # some request was admitted while others were resident (continuous batching)
    assert any(e[3] > 1 for e in admits)
    # and admission happened between retirements, not only at the start
    first_retire = min(e[2] for e in gpu.log if e[0] == "retire")
    assert any(e[2] > first_retire for e in admits)


def test_budget_is_respected_under_overload():
    gpu = FakeGPU(step_cost=0.05)
    reqs = make_requests(30, seed=2, rate=1000.0)
    sched = Scheduler(budget_bytes=900, max_resident=100, admit=gpu.admit, step=gpu.step, retire=gpu.retire,
                      now=gpu.now, idle_wait=gpu.wait)
    rep = sched.run(reqs)
    assert rep.max_bytes <= 900
    assert rep.completed == 30


def test_request_larger_than_budget_is_rejected():
    gpu = FakeGPU()
    reqs = [Request(0, 0.0, 5, 5000, 100)]
    sched = Scheduler(budget_bytes=1000, max_resident=4, admit=gpu.admit, step=gpu.step, retire=gpu.retire,
                      now=gpu.now, idle_wait=gpu.wait)
    with pytest.raises(ValueError):
        sched.run(reqs)
