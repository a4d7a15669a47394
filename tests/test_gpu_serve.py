"""The serving loop on the GPU: a mixed stream of Gaussian and logistic jobs
that arrive while others run, under a memory budget that forces queueing and
batch rebuilds.  Every job's answer (f_K, eq. (7)) equals, bit for bit, that
of the same job run alone with smc_step -- batched and solo iterations are
identical, and a job's arithmetic does not depend on its neighbours."""
import numpy as np
import pytest
import torch

from paper_1905_10252_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10252_gb300 import build, native

    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    native.lib()
    return native


def make_jobs():
    from paper_1905_10252_gb300.serve import Job, poisson_arrivals

    # arrival order differs from job-id order, so the scheduler's list of
    # active jobs and the batch's member order (sorted ids) differ
    arr = poisson_arrivals(18, rate=400.0, seed=5)[::-1].copy()
    jobs = []
    shapes = inputs.batch_shapes(14, seed=9, n_min=1 << 8, n_max=1 << 14)
    for i, (n, d) in enumerate(shapes):
        mu, sig = inputs.gaussian_target(d, seed=50 + i)
        jobs.append(Job(jid=i, kind="gauss", n=n, d=d, k=7 + (i % 5), seed=100 + i, arrival=float(arr[i]),
                        mu=mu, sigma=sig))
    for i in range(4):
        X, y, _ = inputs.logistic_data(300 + 200 * i, 8, seed=i)
        jobs.append(Job(jid=14 + i, kind="logistic", n=1000 + 700 * i, d=8, k=6, seed=200 + i,
                        arrival=float(arr[14 + i]), X=X, y=y, step=0.1, init_scale=0.5))
    return jobs


def alone(nat, job):
    if job.kind == "gauss":
        s = nat.Sampler(job.n, job.d, dtype=torch.float32, seed=job.seed, mu=job.mu, sigma=job.sigma,
                        step=job.step, init_scale=job.init_scale)
    else:
        s = nat.Sampler(job.n, job.d, dtype=torch.float32, seed=job.seed, target="logistic", X=job.X, y=job.y,
                        prior_var=job.prior_var, step=job.step, init_scale=job.init_scale)
    r = s.step(job.k)
    torch.cuda.synchronize()
    out = r["mean"].cpu().numpy().copy()
    s.close()
    return out


@pytest.mark.parametrize("batched,min_batch", [(True, 1), (True, 4), (False, 1)])
def test_served_results_equal_alone(nat, batched, min_batch):
    """min_batch = 1: every ready Gaussian job goes into the batch; 4: the
    engine alternates between the batch and one launch per job as the number
    of ready jobs changes (the same samplers step both ways)."""
    from paper_1905_10252_gb300.serve import GpuEngine, Scheduler, latency_summary

    jobs = make_jobs()
    eng = GpuEngine(batched=batched, min_batch=min_batch)
    need = sum(eng.bytes_needed(j) for j in jobs)
    sch = Scheduler(eng, budget_bytes=need // 3, round_iters=3)
    done = sch.run(jobs)
    assert len(done) == len(jobs)
    assert sch.rounds > 3
    for j in done:
        assert np.array_equal(j.result, alone(nat, j)), (j.jid, j.kind)
    s = latency_summary(done)
    assert s["p99_s"] >= s["p50_s"] > 0


def test_cancelled_jobs_leave_the_others_unchanged(nat):
    """Jobs cancelled mid-run (resident, in the batch or on their own stream)
    and while queued free their memory; the jobs that finish still give the
    solo answers."""
    from paper_1905_10252_gb300.serve import GpuEngine, Scheduler

    class Canceller(GpuEngine):
        def __init__(self, ids, after):
            super().__init__(batched=True, min_batch=1)
            self.ids, self.after, self.calls, self.sch = ids, after, 0, None

        def step(self, jobs, iters):
            self.calls += 1
            if self.calls == self.after:
                for jid in self.ids:
                    self.sch.cancel(jid)
            return super().step(jobs, iters)

    jobs = make_jobs()
    for j in jobs:
        j.k *= 3  # long enough to be cancelled while resident
    victims = [0, 3, 15, 17]
    eng = Canceller(victims, after=3)
    need = sum(eng.bytes_needed(j) for j in jobs)
    sch = Scheduler(eng, budget_bytes=need // 3, round_iters=3)
    eng.sch = sch
    done = sch.run(jobs)
    assert sorted(j.jid for j in done) == sorted(j.jid for j in jobs if j.jid not in victims)
    assert sorted(j.jid for j in sch.cancelled) == victims
    assert sch.used_bytes == 0 and not eng.samplers and eng.batch is None
    for j in done:
        assert np.array_equal(j.result, alone(nat, j)), (j.jid, j.kind)


def test_served_fp64_job_equals_oracle(nat, orc):
    """One plain FP64 Gaussian job (N = 1024, D = 4, K = 20: the plain
    sampler's configuration) served in the mixed stream, under the memory
    budget, next to batched and logistic jobs: its trajectory is the
    oracle's Algorithm 2 run -- particles, log pi and log w bit for bit, the
    resampling decisions, maxima and survivors of every iteration exactly,
    LSE and log c_t within 1e-10, and f_K within 1e-11."""
    from paper_1905_10252_gb300.serve import GpuEngine, Job, Scheduler

    jobs = make_jobs()
    N, D, K, seed = 1024, 4, 20, 3
    mu, Sigma = inputs.gaussian_target(D, seed=0)
    jobs.append(Job(jid=99, kind="gauss", n=N, d=D, k=K, seed=seed, arrival=float(jobs[5].arrival),
                    mu=mu, sigma=Sigma, step=0.5, init_scale=2.0, dtype="f64", keep=True))
    eng = GpuEngine(batched=True, min_batch=1)
    need = sum(eng.bytes_needed(j) for j in jobs)
    sch = Scheduler(eng, budget_bytes=need // 3, round_iters=3)
    done = {j.jid: j for j in sch.run(jobs)}
    assert len(done) == len(jobs)
    job = done[99]
    ref = orc.run(orc.Target.gauss(mu, Sigma), N, seed, K, init_scale=2.0, step=0.5)
    assert np.array_equal(job.state["x"], ref["x"])
    assert np.array_equal(job.state["logpi"], ref["logpi"])
    assert np.array_equal(job.state["logw"], ref["logw"])
    tr = nat.trace_dicts(torch.as_tensor(job.trace))
    assert len(tr) == K
    for k, rec in enumerate(tr):
        assert rec["t"] == k + 1
        assert rec["resampled"] == int(ref["trace"][k, 4]), k
        assert abs(rec["lse"] - ref["trace"][k, 0]) <= 1e-10, k
        assert abs(rec["logc"] - ref["trace"][k, 1]) <= 1e-10, k
        assert rec["max_logw"] == ref["trace"][k, 3], k
        assert rec["survivors"] == int(ref["trace"][k, 5]), k
    np.testing.assert_allclose(job.result, ref["means"][-1], rtol=0, atol=1e-11)
    # the other jobs still give their solo answers
    for j in done.values():
        if j.jid != 99:
            assert np.array_equal(j.result, alone(nat, j)), (j.jid, j.kind)


@pytest.mark.parametrize("per_class", [1, 4])
def test_slot_engine_results_equal_alone(nat, per_class):
    """The served engine: FP32 Gaussian jobs in a standing batch of slots
    (attached on admission, detached on completion, never rebuilt), under a
    memory budget that forces queueing; with one slot per capacity class
    some jobs find no free slot and run one launch per job.  Every job's
    f_K equals its solo run bit for bit."""
    from paper_1905_10252_gb300.serve import Scheduler, SlotEngine

    jobs = make_jobs()
    eng = SlotEngine(per_class=per_class)
    need = sum(eng.bytes_needed(j) for j in jobs)
    sch = Scheduler(eng, budget_bytes=need // 3, round_iters=3)
    done = sch.run(jobs)
    assert len(done) == len(jobs)
    assert not eng.slot_of and all(len(g["free"]) == len(g["caps"]) for g in eng.groups)
    for j in done:
        assert np.array_equal(j.result, alone(nat, j)), (j.jid, j.kind)
