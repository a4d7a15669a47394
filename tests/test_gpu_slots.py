"""Standing batches of slots (smc_slots_*): samplers attached to fixed-capacity
slots and stepped with a per-slot number of iterations, one launch per stage
for all slots, must give every sampler exactly the results of smc_step on it
alone -- particles, log pi, log w, the per-iteration statistics and f_t --
whatever the other slots hold, whether they idle, and across detach / attach
of other samplers into the same slots (the launch layout is never rebuilt)."""
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


def _bits(t):
    t = t.detach().contiguous()
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu()


def _make(nat, n, d, seed, mode=0):
    mu, sig = inputs.gaussian_target(d, seed=100 + d)
    return nat.Sampler(n, d, dtype=torch.float32, seed=seed, mu=mu, sigma=sig, step=0.4, resample_mode=mode)


def _state(S):
    x, lp = S.current()
    return _bits(x), _bits(lp), _bits(S.logw)


class Job:
    def __init__(self, nat, n, d, seed, k, mode=0):
        self.n, self.d, self.seed, self.k, self.mode = n, d, seed, k, mode
        self.S = _make(nat, n, d, seed, mode)
        self.mean = torch.empty(d, dtype=torch.float64, device="cuda")
        self.trace = torch.zeros(k, nat.STATS_WORDS, dtype=torch.float64, device="cuda")
        self.fhat = torch.empty(d, dtype=torch.float64, device="cuda")
        self.done = 0

    def check_against_solo(self, nat):
        ref = _make(nat, self.n, self.d, self.seed, self.mode)
        r = ref.step(self.k, trace=True, fhat=True)
        ref.sync()
        self.S.sync()
        for u, v in zip(_state(self.S), _state(ref)):
            assert torch.equal(u, v), (self.n, self.d)
        assert torch.equal(_bits(self.mean), _bits(r["mean"]))
        assert torch.equal(_bits(self.fhat), _bits(r["fhat"]))
        assert torch.equal(_bits(self.trace), _bits(r["trace"]))
        ref.close()


def test_slots_equal_solo_with_turnover(nat):
    caps = [1 << 10, 1 << 12, 1 << 14, 1 << 14, 1 << 16, 70000]
    slots = nat.Slots(caps)
    rng = np.random.default_rng(0)
    # (n, d, k, mode) -- uneven sizes within the capacities, every D class
    specs = [(1000, 2, 7, 0), (4096, 8, 11, 1), (9000, 16, 9, 0), (16384, 32, 5, 1), (65536, 16, 8, 0),
             (70000, 5, 6, 1), (777, 3, 4, 1), (3000, 32, 10, 0), (12000, 1, 6, 0), (40000, 12, 7, 1)]
    queue = [Job(nat, n, d, 10 + i, k, mode) for i, (n, d, k, mode) in enumerate(specs)]
    placed = {}
    finished = []
    rounds = 0
    while queue or placed:
        # attach waiting jobs to empty slots that fit them
        for job in list(queue):
            free = [s for s in range(len(caps)) if s not in placed and caps[s] >= job.n]
            if free:
                s = free[0]
                slots.attach(s, job.S, mean=job.mean, trace=job.trace[job.done:], fhat=job.fhat)
                placed[s] = job
                queue.remove(job)
        # per-slot counts: up to 3 iterations, some slots idle this round
        iters = [0] * len(caps)
        for s, job in placed.items():
            if rng.uniform() < 0.8:
                iters[s] = int(min(rng.integers(1, 4), job.k - job.done))
        slots.step(iters)
        for s, job in list(placed.items()):
            job.done += iters[s]
            if job.done == job.k:
                slots.detach(s)
                finished.append(job)
                del placed[s]
        rounds += 1
    slots.sync()
    assert rounds > 5 and len(finished) == len(specs)
    for job in finished:
        job.check_against_solo(nat)
    slots.close()


def test_slots_reject_what_they_cannot_hold(nat):
    slots = nat.Slots([4096, 1024])
    big = _make(nat, 5000, 4, 1)
    with pytest.raises(nat.SmcError) as e:
        slots.attach(0, big)
    assert e.value.code == nat.SMC_EINVAL
    small = _make(nat, 1000, 4, 2)
    slots.attach(1, small)
    other = _make(nat, 500, 4, 3)
    with pytest.raises(nat.SmcError) as e:
        slots.attach(1, other)  # occupied
    assert e.value.code == nat.SMC_EINVAL
    with pytest.raises(nat.SmcError) as e:
        slots.attach(0, small)  # already attached elsewhere
    assert e.value.code == nat.SMC_EINVAL
    mu, sig = inputs.gaussian_target(4, seed=1)
    f64 = nat.Sampler(100, 4, dtype=torch.float64, seed=1, mu=mu, sigma=sig)
    with pytest.raises(nat.SmcError) as e:
        slots.attach(0, f64)
    assert e.value.code == nat.SMC_EINVAL
    with pytest.raises(nat.SmcError) as e:
        slots.step([2, 0])  # iterations for an empty slot
    assert e.value.code == nat.SMC_EINVAL
    slots.step([0, 3])
    slots.detach(1)
    with pytest.raises(nat.SmcError) as e:
        slots.detach(1)
    assert e.value.code == nat.SMC_EINVAL
    slots.sync()
    # the sampler continues on its own after detaching: 3 slot iterations
    # then 2 alone equal 5 alone
    small.step(2)
    ref = _make(nat, 1000, 4, 2)
    ref.step(5)
    for u, v in zip(_state(small), _state(ref)):
        assert torch.equal(u, v)
    slots.close()


def test_slots_many_small_jobs_one_layout(nat):
    """A few hundred short jobs through 32 slots of mixed capacity (the
    serving pattern): every result equals its solo run."""
    caps = [1 << c for c in (10, 11, 12, 13, 14, 15, 16, 17)] * 4
    slots = nat.Slots(caps)
    shapes = inputs.batch_shapes(120, seed=3, n_min=1 << 9, n_max=1 << 17)
    jobs = [Job(nat, int(n), int(d), 500 + i, 3 + i % 4, 0) for i, (n, d) in enumerate(shapes)]
    queue, placed, finished = list(jobs), {}, []
    while queue or placed:
        for job in list(queue):
            free = [s for s in range(len(caps)) if s not in placed and caps[s] >= job.n]
            if free:
                s = min(free, key=lambda q: caps[q])
                slots.attach(s, job.S, mean=job.mean, trace=job.trace[job.done:], fhat=job.fhat)
                placed[s] = job
                queue.remove(job)
        iters = [0] * len(caps)
        for s, job in placed.items():
            iters[s] = min(2, job.k - job.done)
        slots.step(iters)
        for s, job in list(placed.items()):
            job.done += iters[s]
            if job.done == job.k:
                slots.detach(s)
                finished.append(job)
                del placed[s]
    slots.sync()
    assert len(finished) == len(jobs)
    for job in finished[::7]:
        job.check_against_solo(nat)
    for job in finished:
        job.S.close()
    slots.close()
