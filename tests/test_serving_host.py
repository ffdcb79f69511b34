"""Host logic of the serving loop (no GPU): FIFO admission under a memory budget,
continuous batching (requests join while others are resident), rejection of requests that
can never fit, eviction of requests whose admission or read-back fails, and latency
bookkeeping, on a simulated clock.  The fake device below does what the library's
apic_batch_admit / apic_batch_run do: refuse a member over the budget, step to the nearest
completion, hand back the finished members."""
import numpy as np
import pytest

from paper_1603_06188_gb300.serving import Deferred, Request, Scheduler, poisson_arrivals


class FakeGPU:
    """Each batched step costs `step_cost` seconds of simulated time; admission is free."""

    def __init__(self, budget, step_cost=0.01, fail_admit=(), fail_retire=()):
        self.t = 0.0
        self.budget = budget
        self.step_cost = step_cost
        self.resident = {}
        self.left = {}
        self.steps_done = {}
        self.log = []
        self.fail_admit = set(fail_admit)
        self.fail_retire = set(fail_retire)

    def now(self):
        return self.t

    def resident_bytes(self):
        return sum(r.footprint for r in self.resident.values())

    def admit(self, r):
        if r.rid in self.fail_admit:
            raise RuntimeError("admission failed")
        if self.resident_bytes() + r.footprint > self.budget:
            raise Deferred()
        self.resident[r.rid] = r
        self.left[r.rid] = r.steps
        self.steps_done[r.rid] = 0
        self.log.append(("admit", r.rid, self.t, len(self.resident)))
        return r.rid

    def run(self, n):
        k = min([n] + list(self.left.values()))
        for rid in self.resident:
            self.steps_done[rid] += k
            self.left[rid] -= k
        self.t += k * self.step_cost
        done = [rid for rid in self.resident if self.left[rid] == 0]
        for rid in done:
            del self.resident[rid]
            del self.left[rid]
        return done, k

    def retire(self, r, h):
        assert self.steps_done[r.rid] == r.steps, "a simulation must get exactly its steps"
        self.log.append(("retire", r.rid, self.t, len(self.resident)))
        if r.rid in self.fail_retire:
            raise RuntimeError("read-back failed")

    def wait(self, dt):
        self.t += max(dt, 1e-6)


def make_requests(n, seed=0, rate=50.0):
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(rng, rate, n)
    return [Request(i, float(arr[i]), int(rng.integers(5, 40)), int(rng.integers(1, 10)) * 100, int(rng.integers(1000, 5000)))
            for i in range(n)]


def scheduler(gpu, budget, max_resident, max_chunk=8):
    return Scheduler(budget_bytes=budget, max_resident=max_resident, admit=gpu.admit, run=gpu.run,
                     retire=gpu.retire, now=gpu.now, resident_bytes=gpu.resident_bytes, max_chunk=max_chunk,
                     idle_wait=gpu.wait)


def test_every_request_gets_exactly_its_steps_and_latency_is_recorded():
    gpu = FakeGPU(2000)
    reqs = make_requests(60)
    rep = scheduler(gpu, 2000, 8, max_chunk=4).run(reqs)
    assert rep.completed == 60
    assert len(rep.latencies) == 60
    assert all(r.finished >= r.admitted >= r.arrival for r in reqs)
    assert rep.particle_steps == sum(r.particles * r.steps for r in reqs)
    assert rep.max_bytes <= 2000 and rep.max_resident <= 8
    assert rep.percentile(99) >= rep.percentile(50) > 0
    assert not rep.rejected and not rep.failed


def test_admission_is_fifo_and_continuous():
    gpu = FakeGPU(1500)
    reqs = make_requests(40, seed=1, rate=200.0)
    scheduler(gpu, 1500, 6).run(reqs)
    admits = [e for e in gpu.log if e[0] == "admit"]
    assert [e[1] for e in admits] == sorted(e[1] for e in admits)      # arrival order kept
    # some request was admitted while others were resident (continuous batching)
    assert any(e[3] > 1 for e in admits)
    # and admission happened between retirements, not only at the start
    first_retire = min(e[2] for e in gpu.log if e[0] == "retire")
    assert any(e[2] > first_retire for e in admits)


def test_budget_is_respected_under_overload():
    gpu = FakeGPU(900, step_cost=0.05)
    reqs = make_requests(30, seed=2, rate=1000.0)
    rep = scheduler(gpu, 900, 100).run(reqs)
    assert rep.max_bytes <= 900
    assert rep.completed == 30


def test_request_larger_than_budget_is_rejected_at_arrival_and_others_are_served():
    """One request that can never fit, in the middle of a stream: it is rejected when it
    arrives, it blocks nobody behind it, and every other request completes."""
    gpu = FakeGPU(1000)
    reqs = make_requests(20, seed=3, rate=100.0)
    big = reqs[10]
    big.footprint = 5000
    rep = scheduler(gpu, 1000, 8).run(reqs)
    assert rep.rejected == [big.rid]
    assert rep.completed == 19
    assert big.admitted < 0 and big.finished < 0
    # requests that arrived after it joined a non-empty batch: nothing waited for the
    # batch to drain behind it
    later = {r.rid for r in reqs if r.arrival > big.arrival}
    assert any(e[1] in later and e[3] > 1 for e in gpu.log if e[0] == "admit")


def test_failing_requests_are_evicted_and_serving_continues():
    gpu = FakeGPU(2000, fail_admit={3, 17}, fail_retire={8})
    reqs = make_requests(30, seed=4)
    rep = scheduler(gpu, 2000, 8).run(reqs)
    assert sorted(rid for rid, _ in rep.failed) == [3, 8, 17]
    assert rep.completed == 27
    assert all(r.finished > 0 for r in reqs if r.rid not in (3, 8, 17))


def test_only_oversize_requests_cannot_wait_forever():
    gpu = FakeGPU(1000)
    reqs = [Request(0, 0.0, 5, 5000, 100), Request(1, 0.0, 5, 400, 100)]
    rep = scheduler(gpu, 1000, 4).run(reqs)
    assert rep.rejected == [0] and rep.completed == 1
