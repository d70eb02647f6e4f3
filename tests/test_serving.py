"""The serving loop (continuous batching) on the CPU, against a fake batch.

The fake stands in for ncorp_batch: it keeps the admitted disks, refuses a
disk that would take its memory over the budget (as the batch does with
NCORP_ENOMEM), counts every disk's steps and advances a simulated clock by a
cost per step.  The tests check that every request gets exactly its steps,
that requests arriving while others run join them (the work overlaps), that
admission follows arrival order and never exceeds the budget, and the
latency figures on a case worked out by hand.
"""
import numpy as np
import pytest

from paper_2310_20374_gb300 import serving


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, s):
        self.t += s


class FakeBatch:
    def __init__(self, clock, budget=None, bytes_per_moonlet=1000, step_s=lambda moonlets: 1e-3 + 1e-8 * moonlets):
        self.clock, self.budget, self.bpm, self.step_s = clock, budget, bytes_per_moonlet, step_s
        self.disks = {}        # id -> [request, steps done]
        self.next = 0
        self.used = self.peak = 0
        self.admitted = []     # request arrival times in admission order
        self.max_disks = 0

    def add(self, req):
        need = self.bpm * req.n
        if self.budget is not None and self.used + need > self.budget:
            raise serving.BudgetFull("budget")
        self.used += need
        self.peak = max(self.peak, self.used)
        did = self.next
        self.next += 1
        self.disks[did] = [req, 0]
        self.admitted.append(req.arrival)
        return did

    def run(self, k):
        assert self.disks
        self.clock.t += k * self.step_s(sum(r.n for r, _ in self.disks.values()))
        for v in self.disks.values():
            v[1] += k
        self.max_disks = max(self.max_disks, len(self.disks))

    def evict(self, req):
        r, done = self.disks.pop(req.disk_id)
        assert r is req and done == 0        # only disks that were never stepped go back to the queue
        self.used -= self.bpm * req.n

    def finish(self, req, out=None):
        r, done = self.disks.pop(req.disk_id)
        assert r is req and done == req.steps   # exactly the steps asked for, never more
        self.used -= self.bpm * req.n


def run(reqs, **kw):
    clock = Clock()
    fb = FakeBatch(clock, **{k: v for k, v in kw.items() if k in ("budget", "step_s")})
    st = serving.serve(fb, reqs, clock=clock, sleep=clock.sleep,
                       **{k: v for k, v in kw.items() if k in ("tick_steps", "max_wall")})
    return st, fb


def test_every_request_gets_its_steps_and_work_overlaps():
    reqs = serving.poisson_requests(20.0, 5.0, 1e3, 1e5, (3, 4, 6), 100, seed=1)
    st, fb = run(reqs, tick_steps=10)
    assert st["served"] == st["requests"] == len(reqs) and not fb.disks
    assert st["moonlet_steps"] == sum(r.n * 100 for r in reqs)
    assert fb.max_disks >= 2 and st["concurrent_disks_max"] >= 2
    # some request was admitted while an earlier one was still running
    assert any(b.admitted < a.done for a in reqs for b in reqs if b.arrival > a.arrival)
    assert all(r.admitted >= r.arrival and r.done > r.admitted for r in reqs)


def test_admission_in_arrival_order_within_the_budget():
    reqs = serving.poisson_requests(50.0, 2.0, 1e3, 1e5, (3, 6), 30, seed=2)
    budget = 1000 * 150000   # room for a few disks at a time
    st, fb = run(reqs, tick_steps=5, budget=budget)
    assert st["served"] == len(reqs)
    assert fb.peak <= budget
    assert fb.admitted == sorted(fb.admitted)            # first come, first admitted
    assert st["admission_wait_s_p99"] > 0.0               # the budget made some requests wait


def test_a_disk_larger_than_the_budget_alone_is_an_error():
    reqs = [serving.Request(arrival=0.0, n=5000, p=3, steps=10)]
    with pytest.raises(RuntimeError, match="does not fit"):
        run(reqs, budget=1000 * 4999)


def test_latencies_of_a_worked_example():
    # A arrives at 0 (20 steps), B at 0.5 (10 steps); every step of the batch takes 0.1 s.
    # tick 1: [0, 1.0] A alone, 10 steps; B admitted at 1.0 (waited 0.5 s);
    # tick 2: [1.0, 2.0] A and B, 10 steps: both finish at 2.0.
    reqs = [serving.Request(arrival=0.0, n=1000, p=3, steps=20), serving.Request(arrival=0.5, n=1000, p=3, steps=10)]
    st, _ = run(reqs, tick_steps=10, step_s=lambda moonlets: 0.1)
    assert st["ticks"] == 2 and st["batch_steps"] == 20
    assert st["tick_ms_p50"] == pytest.approx(1000.0) and st["tick_ms_p99"] == pytest.approx(1000.0)
    assert st["step_ms_p50"] == pytest.approx(100.0) and st["step_ms_p99"] == pytest.approx(100.0)
    assert reqs[0].done == pytest.approx(2.0) and reqs[1].done == pytest.approx(2.0)
    assert reqs[1].admitted == pytest.approx(1.0)
    assert st["request_s_p50"] == pytest.approx(np.percentile([2.0, 1.5], 50))
    assert st["admission_wait_s_p99"] == pytest.approx(np.percentile([0.0, 0.5], 99))
    assert st["moonlet_steps"] == 1000 * 30 and st["wall_s"] == pytest.approx(2.0)
    assert st["throughput"] == pytest.approx(15000.0)


def test_ticks_are_shortened_so_no_disk_overshoots():
    reqs = [serving.Request(arrival=0.0, n=100, p=3, steps=7), serving.Request(arrival=0.0, n=100, p=3, steps=23)]
    st, _ = run(reqs, tick_steps=10)
    assert st["served"] == 2          # finish() asserts the exact step counts
    assert st["ticks"] == 3           # 7 (both), then 10 and 6 (the second alone): 7 + 10 + 6 = 23
    assert st["batch_steps"] == 23


def test_admission_stops_at_the_end_of_the_window():
    reqs = serving.poisson_requests(10.0, 10.0, 1e3, 1e4, (3,), 10, seed=3)
    st, _ = run(reqs, tick_steps=10, max_wall=3.0)
    assert 0 < st["served"] < len(reqs)
    assert all(r.admitted is None or r.admitted <= 3.0 + 1e-9 for r in reqs)


class TightBatch(FakeBatch):
    """A fake batch whose runs fail (stepping nothing) while its disks hold more than `run_limit`, as a
    real batch does when it cannot lay out its forests in device memory."""

    def __init__(self, clock, run_limit, **kw):
        super().__init__(clock, **kw)
        self.run_limit, self.failed_runs = run_limit, 0

    def run(self, k):
        if self.used > self.run_limit:
            self.failed_runs += 1
            raise serving.BudgetFull("run")
        super().run(k)


def test_a_run_that_does_not_fit_sends_the_newest_admissions_back():
    clock = Clock()
    reqs = [serving.Request(arrival=0.0, n=1000, p=3, steps=20) for i in range(8)]
    fb = TightBatch(clock, run_limit=1000 * 1000 * 3)   # three disks fit a run, more are admitted
    st = serving.serve(fb, reqs, tick_steps=5, clock=clock, sleep=clock.sleep)
    assert st["served"] == len(reqs) and fb.failed_runs > 0   # finish() checked the exact step counts
    assert fb.max_disks <= 3
    assert all(r.done > r.admitted >= r.arrival for r in reqs)


def test_a_disk_that_no_run_fits_is_an_error():
    clock = Clock()
    fb = TightBatch(clock, run_limit=10)
    with pytest.raises(RuntimeError, match="on its own"):
        serving.serve(fb, [serving.Request(arrival=0.0, n=1000, p=3, steps=5)], clock=clock, sleep=clock.sleep)


def test_progress_reports_every_run_and_tick():
    reqs = [serving.Request(arrival=0.0, n=1000, p=3, steps=20), serving.Request(arrival=0.5, n=1000, p=3, steps=10)]
    clock, seen = Clock(), []
    fb = FakeBatch(clock, step_s=lambda moonlets: 0.1)
    serving.serve(fb, reqs, tick_steps=10, clock=clock, sleep=clock.sleep, progress=seen.append)
    assert [s["event"] for s in seen] == ["run", "tick", "run", "tick"]
    assert [s["disks"] for s in seen] == [1, 1, 2, 0] and seen[-1]["served"] == 2
    assert seen[1]["t"] == pytest.approx(1.0) and seen[2]["moonlets"] == 2000 and seen[-1]["ticks"] == 2
