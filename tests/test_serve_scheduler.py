"""Host logic of the serving loop (paper_1905_10252_gb300/serve.py) with a fake
engine and a fake clock: admission within the memory budget, first fit in
arrival order with the no-overtaking rule for jobs that waited too long,
every job run for exactly its K iterations, latency accounting."""
import math

import numpy as np
import pytest

from paper_1905_10252_gb300.serve import Engine, Job, Scheduler, latency_summary, poisson_arrivals


class FakeClock:
    def __init__(self, dt=0.001):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeEngine(Engine):
    def __init__(self):
        self.resident = {}
        self.max_used = 0
        self.admitted_order = []
        self.iters = {}

    def bytes_needed(self, job):
        return job.n

    def admit(self, job):
        self.resident[job.jid] = job.n
        self.max_used = max(self.max_used, sum(self.resident.values()))
        self.admitted_order.append(job.jid)
        self.iters[job.jid] = 0

    def step(self, jobs, iters):
        for j in jobs:
            assert 1 <= iters[j.jid] <= j.k - j.done_iters
            self.iters[j.jid] += iters[j.jid]
        self.pending = [j.jid for j in jobs]
        return list(self.pending)

    def completed(self, block=True):
        out, self.pending = self.pending, []
        return out

    def result(self, job):
        return np.array([float(self.iters[job.jid])])

    def release(self, job):
        del self.resident[job.jid]


def make_jobs(ns, ks, arrivals):
    return [Job(jid=i, kind="gauss", n=n, d=2, k=k, seed=i, arrival=a) for i, (n, k, a) in
            enumerate(zip(ns, ks, arrivals))]


def test_budget_respected_and_every_job_runs_k_iterations():
    g = np.random.default_rng(0)
    ns = g.integers(10, 400, size=200)
    ks = g.integers(1, 23, size=200)
    arr = poisson_arrivals(200, rate=500.0, seed=1)
    eng = FakeEngine()
    sch = Scheduler(eng, budget_bytes=1000, round_iters=4, clock=FakeClock())
    done = sch.run(make_jobs(ns, ks, arr))
    assert len(done) == 200
    assert eng.max_used <= 1000
    for j in done:
        assert j.done_iters == j.k and float(j.result[0]) == j.k
        assert j.arrival <= j.admitted <= j.finished
    assert sch.used_bytes == 0 and not eng.resident


def test_small_job_overtakes_a_large_one_that_does_not_fit():
    # job 0 fills the budget; job 1 (large) must wait; job 2 (small) fits beside job 0
    jobs = make_jobs([700, 600, 200], [50, 5, 5], [0.0, 0.0, 0.0])
    eng = FakeEngine()
    Scheduler(eng, budget_bytes=1000, round_iters=5, clock=FakeClock()).run(jobs)
    assert eng.admitted_order == [0, 2, 1]


def test_long_waiting_job_blocks_overtaking():
    # job 1 cannot fit while job 0 runs; after max_wait_rounds it blocks job 2..
    jobs = make_jobs([700, 600, 200, 200], [60, 5, 5, 5], [0.0, 0.0, 0.0, 0.0005])
    eng = FakeEngine()
    Scheduler(eng, budget_bytes=1000, round_iters=1, max_wait_rounds=3, clock=FakeClock(dt=0.01)).run(jobs)
    # job 2 was admitted at once (job 1 had not yet waited long); job 3 arrives
    # after job 1 has waited too long and must come after it
    assert eng.admitted_order.index(1) < eng.admitted_order.index(3)
    assert eng.admitted_order.index(2) < eng.admitted_order.index(1)


def test_job_larger_than_budget_is_rejected():
    eng = FakeEngine()
    with pytest.raises(ValueError):
        Scheduler(eng, budget_bytes=100, clock=FakeClock()).run(make_jobs([101], [1], [0.0]))


def test_latency_summary_and_poisson_stream():
    arr = poisson_arrivals(20000, rate=200.0, seed=3)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 200.0) < 3 * (1 / 200.0) / np.sqrt(20000)
    jobs = make_jobs([1] * 3, [1] * 3, [0.0, 1.0, 2.0])
    for j, lat in zip(jobs, [0.5, 1.0, 3.0]):
        j.finished = j.arrival + lat
    s = latency_summary(jobs)
    assert s["p50_s"] == 1.0 and s["max_s"] == 3.0


class CancellingEngine(FakeEngine):
    """Requests cancellations from inside the serving loop: after `after`
    step calls it cancels the listed ids; release never happens while a
    job's iterations are in flight."""

    def __init__(self, sch_ref, after, ids):
        super().__init__()
        self.sch_ref, self.after, self.ids, self.calls = sch_ref, after, ids, 0
        self.pending = []

    def step(self, jobs, iters):
        self.calls += 1
        if self.calls == self.after:
            for jid in self.ids:
                self.sch_ref[0].cancel(jid)
        return super().step(jobs, iters)

    def release(self, job):
        assert job.jid not in self.pending, "released with iterations in flight"
        super().release(job)


def test_cancel_resident_queued_and_future_jobs():
    # job 0 resident (long), job 1 resident (short), job 2 queued behind the
    # budget, job 3 arrives later; cancel 0, 2 and 3 after the second round
    jobs = make_jobs([400, 400, 500, 100], [100, 10, 5, 5], [0.0, 0.0, 0.0, 1.0])
    ref = [None]
    eng = CancellingEngine(ref, after=2, ids=[0, 2, 3])
    sch = Scheduler(eng, budget_bytes=1000, round_iters=5, clock=FakeClock())
    ref[0] = sch
    done = sch.run(jobs)
    assert [j.jid for j in done] == [1]
    assert sorted(j.jid for j in sch.cancelled) == [0, 2, 3]
    by = {j.jid: j for j in jobs}
    assert by[0].status == "cancelled" and by[0].result is None and 0 < by[0].done_iters < 100
    assert by[2].status == "cancelled" and math.isnan(by[2].admitted)  # never admitted
    assert by[3].status == "cancelled" and by[3].done_iters == 0
    assert by[1].status == "done" and by[1].done_iters == 10
    assert sch.used_bytes == 0 and not eng.resident
    assert not sch._cancel_ids


def test_cancelling_a_finished_job_changes_nothing():
    jobs = make_jobs([100], [5], [0.0])
    eng = FakeEngine()
    sch = Scheduler(eng, budget_bytes=1000, clock=FakeClock())
    done = sch.run(jobs)
    sch.cancel(0)
    assert done[0].status == "done" and float(done[0].result[0]) == 5 and not sch.cancelled


def test_deadline_cancels_jobs_that_would_finish_late():
    # one slot: the first job runs 200 iterations (one round = 5 iterations =
    # a few clock ticks), the others wait; a short deadline cancels the waiters
    jobs = make_jobs([900, 900, 900], [200, 5, 5], [0.0, 0.0, 0.0])
    jobs[1].deadline = 0.01
    eng = FakeEngine()
    sch = Scheduler(eng, budget_bytes=1000, round_iters=5, clock=FakeClock())
    done = sch.run(jobs)
    assert sorted(j.jid for j in done) == [0, 2]
    assert [j.jid for j in sch.cancelled] == [1]
    assert jobs[1].finished - jobs[1].arrival > 0.01
    assert sch.used_bytes == 0 and not eng.resident


def test_admission_is_spread_over_passes():
    """At most admit_per_pass jobs are admitted per pass of the loop (so that
    launches start while the rest are admitted); every job still runs."""
    class Counting(FakeEngine):
        def __init__(self):
            super().__init__()
            self.steps = []

        def step(self, jobs, iters):
            self.steps.append(len(self.resident))
            return super().step(jobs, iters)

    eng = Counting()
    jobs = make_jobs([1] * 50, [3] * 50, [0.0] * 50)
    sch = Scheduler(eng, budget_bytes=10 ** 6, round_iters=1, admit_per_pass=8)
    done = sch.run(jobs)
    assert len(done) == 50
    assert eng.steps[0] == 8  # the first launch came after 8 admissions
    assert max(eng.steps) <= 50
