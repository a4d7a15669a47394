"""Serving many sampler jobs on one GPU with continuous batching.

A job is one SMC run (Algorithm 2 for K iterations) of its own target, N and
D; its answer is the weighted mean f_K of eq. (7).  The server keeps every
admitted job's particles, weights, log-targets and RNG counter (the iteration
index t, the Philox key is the job's seed) resident in HBM, and advances all
resident jobs together in rounds of a few iterations:

  * Gaussian FP32 jobs share one batched launch per stage (``native.Batch``,
    one CUDA graph of the batched iteration) when at least ``min_batch`` of
    them are ready together; the batch is rebuilt whenever jobs join or
    leave, between rounds.  Fewer ready jobs (light load, or arrivals while
    the batch runs) take one launch per job on their own streams, which
    starts them at once instead of waiting for the batch's round;
  * logistic-regression jobs run their own iterations (tensor-core
    likelihood) on their own streams, concurrently with the batch;
  * Gaussian work runs on high-priority streams, so that its short kernels
    are scheduled between the long logistic ones (shortest job first).

Jobs that arrive while others are on the GPU wait in a queue and are admitted
as soon as their device memory fits in the budget (first fit in arrival
order: a small job may pass a large one that does not fit yet, but a job that
has waited longer than ``max_wait_rounds`` rounds blocks everything behind it
until it is admitted).  A job's results do not depend on the jobs around it:
batched and solo iterations are bit-identical (tests/test_gpu_serve.py).

A job can be cancelled, by ``Scheduler.cancel`` (from any thread) or by its
own ``deadline`` (seconds after arrival): a queued job leaves the queue; a
resident one is released as soon as the iterations already launched for it
have completed (no kernel is interrupted), and its memory returns to the
budget.  Cancelled jobs end in ``Scheduler.cancelled`` with no result.

The scheduling policy (``Scheduler``) is plain host logic over an ``Engine``
interface, so it is tested on the CPU with a fake engine; ``GpuEngine`` is the
CUDA implementation.  Nothing here computes any part of the sampler.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    """One sampler run: kind 'gauss' (mu, sigma) or 'logistic' (X, y);
    dtype 'f32' (every kind) or 'f64' (Gaussian jobs, one launch per job).
    keep = True also keeps the per-iteration statistics (``trace``) and the
    final particles, log pi and log w (``state``) for inspection."""

    jid: int
    kind: str
    n: int
    d: int
    k: int
    seed: int
    arrival: float = 0.0           # seconds since the start of the stream
    mu: np.ndarray | None = None
    sigma: np.ndarray | None = None
    X: np.ndarray | None = None
    y: np.ndarray | None = None
    prior_var: float = 4.0
    step: float = 0.5
    init_scale: float = 2.0
    deadline: float = math.inf     # cancelled if not finished this long after arrival
    dtype: str = "f32"
    keep: bool = False
    # filled in by the scheduler
    admitted: float = math.nan
    finished: float = math.nan
    done_iters: int = 0
    result: np.ndarray | None = None
    trace: np.ndarray | None = None  # (keep) K statistics records
    state: dict | None = None        # (keep) final x, logpi, logw
    waited_rounds: int = 0
    status: str = "new"            # queued, resident, done or cancelled

    @property
    def m(self) -> int:
        return 0 if self.X is None else int(self.X.shape[0])

    def latency(self) -> float:
        return self.finished - self.arrival


class Engine:
    """What the scheduler needs from a device (see GpuEngine)."""

    def bytes_needed(self, job: Job) -> int:
        raise NotImplementedError

    def admit(self, job: Job) -> None:
        raise NotImplementedError

    def step(self, jobs: list[Job], iters: dict[int, int]) -> list[int]:
        """Launches iters[job.jid] iterations of jobs (asynchronously) and
        returns the ids it launched (the others stay idle for now)."""
        raise NotImplementedError

    def completed(self, block: bool = True) -> list[int]:
        """Ids of jobs whose launched iterations have all completed since the
        last call; with block, waits until at least one has, when any work
        is pending."""
        raise NotImplementedError

    def result(self, job: Job) -> np.ndarray:
        raise NotImplementedError

    def release(self, job: Job) -> None:
        raise NotImplementedError


@dataclass
class Scheduler:
    engine: Engine
    budget_bytes: int
    round_iters: int = 5
    max_wait_rounds: int = 50
    admit_per_pass: int = 32       # jobs admitted per pass of the loop, so that launches start early
    clock: callable = time.perf_counter
    queue: list[Job] = field(default_factory=list)
    active: list[Job] = field(default_factory=list)
    finished: list[Job] = field(default_factory=list)
    cancelled: list[Job] = field(default_factory=list)
    used_bytes: int = 0
    rounds: int = 0
    _cancel_ids: set = field(default_factory=set)
    _lock: threading.Lock = field(default_factory=threading.Lock)
    _capped: bool = False          # the last admission pass stopped at admit_per_pass

    def cancel(self, jid: int) -> None:
        """Requests the cancellation of job jid (takes effect in the serving
        loop; a job that has already finished is left as it is)."""
        with self._lock:
            self._cancel_ids.add(int(jid))

    def _take_cancels(self, now: float, busy: dict[int, int]) -> None:
        with self._lock:
            ids = set(self._cancel_ids)
        ids |= {j.jid for j in self.queue + self.active if now - j.arrival > j.deadline}
        if not ids:
            return
        keep_q = []
        for j in self.queue:
            if j.jid in ids:
                self._drop(j, now)
            else:
                keep_q.append(j)
        self.queue = keep_q
        keep_a = []
        for j in self.active:
            if j.jid in ids and j.jid not in busy:  # nothing of it in flight
                self.engine.release(j)
                self.used_bytes -= self.engine.bytes_needed(j)
                self._drop(j, now)
            else:
                keep_a.append(j)
        self.active = keep_a
        # requests for jobs that have ended are spent; those for jobs not yet
        # arrived, or with iterations in flight, stay
        ended = {j.jid for j in self.cancelled} | {j.jid for j in self.finished}
        with self._lock:
            self._cancel_ids -= ended

    def _drop(self, job: Job, now: float) -> None:
        job.status = "cancelled"
        job.finished = now
        job.result = None
        self.cancelled.append(job)

    def _admit(self, now: float) -> None:
        blocked = False
        still = []
        admitted = 0
        self._capped = False
        for job in self.queue:
            if admitted >= self.admit_per_pass:
                still.append(job)  # (considered again at the next pass)
                self._capped = True
                continue
            need = self.engine.bytes_needed(job)
            if need > self.budget_bytes:
                raise ValueError(f"job {job.jid} needs {need} bytes, more than the whole budget")
            if not blocked and self.used_bytes + need <= self.budget_bytes:
                self.engine.admit(job)
                job.admitted = now
                job.status = "resident"
                self.used_bytes += need
                self.active.append(job)
                admitted += 1
            else:
                job.waited_rounds += 1
                still.append(job)
                if job.waited_rounds > self.max_wait_rounds:
                    blocked = True  # no overtaking a job that has waited too long
        self.queue = still

    def run(self, jobs: list[Job], t0: float | None = None) -> list[Job]:
        """Serves jobs (sorted by arrival); arrivals are released by the
        clock.  A job gets new iterations as soon as its previous ones have
        completed, so short and long jobs progress independently."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        start = self.clock() if t0 is None else t0
        busy: dict[int, int] = {}
        i = 0
        while i < len(pending) or self.queue or self.active:
            now = self.clock() - start
            while i < len(pending) and pending[i].arrival <= now:
                pending[i].status = "queued"
                self.queue.append(pending[i])
                i += 1
            self._take_cancels(now, busy)
            self._admit(now)
            idle = [j for j in self.active if j.jid not in busy]
            if idle:
                iters = {j.jid: min(self.round_iters, j.k - j.done_iters) for j in idle}
                launched = self.engine.step(idle, iters)
                busy.update({jid: iters[jid] for jid in launched})
                self.rounds += 1 if launched else 0
            if not busy:
                if i < len(pending):  # idle until the next arrival
                    wait = pending[i].arrival - (self.clock() - start)
                    if wait > 0:
                        time.sleep(min(wait, 0.005))
                continue
            # (jobs left queued by the per-pass cap: admit them without
            # waiting for a completion)
            done_ids = set(self.engine.completed(block=not self._capped))
            still = []
            for j in self.active:
                if j.jid in done_ids:
                    j.done_iters += busy.pop(j.jid)
                if j.done_iters >= j.k:
                    j.result = self.engine.result(j)
                    j.finished = self.clock() - start
                    j.status = "done"
                    self.engine.release(j)
                    self.used_bytes -= self.engine.bytes_needed(j)
                    self.finished.append(j)
                else:
                    still.append(j)
            self.active = still
        return self.finished


def latency_summary(jobs: list[Job]) -> dict:
    lat = np.array([j.latency() for j in jobs])
    return {"jobs": len(jobs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times of a Poisson stream (exponential gaps, mean 1 / rate)."""
    g = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5E7]))
    return np.cumsum(g.exponential(1.0 / rate, size=count))


_STREAMS: dict = {}  # (device, priority) -> streams free for reuse by new jobs


class _DeviceCopies:
    """Device copies of the host arrays jobs bring (targets, data), made once
    per array: a cache entry keeps its array alive, so its id() stays unique
    while cached (least recently used entries dropped beyond ``size``)."""

    def __init__(self, torch, device, size: int = 256):
        self.torch, self.device, self.size = torch, device, size
        self.entries: dict = {}

    def get(self, a, dtype):
        if a is None:
            return None
        key = (id(a), dtype)
        hit = self.entries.pop(key, None)
        if hit is None:
            hit = (a, self.torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(self.device))
        self.entries[key] = hit  # most recent last
        while len(self.entries) > self.size:
            self.entries.pop(next(iter(self.entries)))
        return hit[1]


class GpuEngine(Engine):
    """Jobs as libsmc samplers on one GPU (see the module docstring)."""

    def __init__(self, batched: bool = True, device: str = "cuda", min_batch: int = 16):
        import torch

        from . import native

        self.torch, self.native = torch, native
        self.batched = batched
        self.min_batch = max(1, int(min_batch))
        self.device = device
        self.samplers: dict[int, object] = {}
        self.means: dict[int, object] = {}
        self.traces: dict[int, object] = {}
        self.batch = None
        self.batch_ids: tuple = ()
        # short jobs first: Gaussian work (the batch, or each Gaussian job in
        # one-per-launch mode) runs on high-priority streams, so that its small
        # kernels are scheduled between the long logistic likelihood kernels
        lo_prio, hi_prio = torch.cuda.Stream.priority_range()
        self.hi_prio = hi_prio
        self.stream = torch.cuda.Stream(device=device, priority=hi_prio)
        self.pending: list = []  # (event, job ids, is the batch) of launched work
        self.batch_busy = False
        self.copies = _DeviceCopies(torch, device)
        self.job_stream: dict[int, object] = {}

    def _stream(self, job: Job):
        """A stream of its own for the job, reused from released jobs."""
        key = (str(self.device), self.hi_prio if job.kind == "gauss" else 0)
        pool = _STREAMS.setdefault(key, [])
        st = pool.pop() if pool else self.torch.cuda.Stream(device=self.device, priority=key[1])
        self.job_stream[job.jid] = (key, st)
        return st

    def bytes_needed(self, job: Job) -> int:
        # particle state (two buffers), log w, two log pi buffers, workspace
        # (its logistic data included) and the batch's per-member arguments
        es = 8 if job.dtype == "f64" else 4
        ws = 2 * job.n * job.d * es + job.n * 8 + 2 * job.n * es
        ws += 32 * job.n + 12 * job.n + 64 * job.d * job.d + (1 << 16)
        ws += min(304, -(-job.n // 128)) * job.d * (job.d + 1) // 2 * 8  # covariance partials
        if job.kind == "logistic":
            m_pad = (job.m + 255) // 256 * 256
            ws += job.m * job.d * 4 + job.m * 4 + m_pad * 128
        return int(ws)

    def admit(self, job: Job) -> None:
        nat = self.native
        torch = self.torch
        if job.kind == "gauss":
            dt = torch.float64 if job.dtype == "f64" else torch.float32
            s = nat.Sampler(job.n, job.d, dtype=dt, seed=job.seed, mu=self.copies.get(job.mu, torch.float64),
                            sigma=self.copies.get(job.sigma, torch.float64), step=job.step,
                            init_scale=job.init_scale, stream=self._stream(job))
        else:
            s = nat.Sampler(job.n, job.d, dtype=torch.float32, seed=job.seed, target="logistic",
                            X=self.copies.get(job.X, torch.float32), y=self.copies.get(job.y, torch.float32),
                            prior_var=job.prior_var, step=job.step, init_scale=job.init_scale,
                            stream=self._stream(job))
        self.samplers[job.jid] = s
        self.means[job.jid] = self.torch.empty(job.d, dtype=self.torch.float64, device=self.device)
        if job.keep:
            self.traces[job.jid] = self.torch.zeros(max(job.k, 1), nat.STATS_WORDS, dtype=self.torch.float64,
                                                    device=self.device)

    def _trace_ptr(self, job: Job):
        """Device address of the job's trace record for its next iteration
        (smc_step writes one record per iteration from there)."""
        tr = self.traces.get(job.jid)
        return None if tr is None else tr[job.done_iters:].data_ptr()

    def _batch_for(self, jobs: list[Job]):
        ids = tuple(sorted(j.jid for j in jobs))
        if ids != self.batch_ids:
            if self.batch is not None:
                self.batch.sync()
                self.batch.close()
            self.batch = self.native.Batch([self.samplers[i] for i in ids], stream=self.stream) if ids else None
            self.batch_ids = ids
        return self.batch

    def step(self, jobs: list[Job], iters: dict[int, int]) -> list[int]:
        nat = self.native
        L = nat.lib()
        torch = self.torch
        # FP32 Gaussian jobs can share the batched launch; FP64 and logistic
        # jobs take one launch per job
        gauss = [j for j in jobs if j.kind == "gauss" and j.dtype == "f32" and not j.keep]
        others = [j for j in jobs if j not in gauss]
        launched = []
        if self.batched and gauss and not self.batch_busy and len(gauss) >= self.min_batch:
            # the batch advances every member by the same count: jobs needing
            # fewer iterations this round (their last) step alone
            k = min(iters[j.jid] for j in gauss)
            full = [j for j in gauss if iters[j.jid] == k]
            rest = [j for j in gauss if iters[j.jid] != k]
            b = self._batch_for(full)
            # members may have stepped alone since the batch was built: its
            # stream waits for their streams
            for i in self.batch_ids:
                self.stream.wait_stream(self.samplers[i].stream)
            # outputs in the batch's member order
            b.step_raw(k, means=[self.means[i] for i in self.batch_ids])
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.pending.append((ev, [j.jid for j in full], True))
            self.batch_busy = True
            launched += [j.jid for j in full]
            others = rest + others
        elif gauss:
            others = gauss + others
        for j in others:
            s = self.samplers[j.jid]
            s.stream.wait_stream(torch.cuda.current_stream(self.device))
            nat._check(L.smc_step(s.h, int(iters[j.jid]), nat._ptr(self.means[j.jid]), None, self._trace_ptr(j),
                                  None), s.h)
            ev = torch.cuda.Event()
            ev.record(s.stream)
            self.pending.append((ev, [j.jid], False))
            launched.append(j.jid)
        return launched

    def completed(self, block: bool = True) -> list[int]:
        if not self.pending:
            return []
        # poll every launch, with a short sleep between polls: blocking on any
        # one event would hold up the relaunch of the others (and the
        # admission of arrivals) until it completes
        while True:
            done = [p for p in self.pending if p[0].query()]
            if done or not block:
                break
            time.sleep(20e-6)
        self.pending = [p for p in self.pending if p not in done]
        if any(p[2] for p in done):
            self.batch_busy = False
        return [jid for _, ids, _ in done for jid in ids]

    def result(self, job: Job) -> np.ndarray:
        if job.keep:
            s = self.samplers[job.jid]
            x, lp = s.current()
            job.state = {"x": x.cpu().numpy().copy(), "logpi": lp.cpu().numpy().copy(),
                         "logw": s.logw.cpu().numpy().copy()}
            job.trace = self.traces[job.jid].cpu().numpy().copy()
        return self.means[job.jid].cpu().numpy().copy()

    def release(self, job: Job) -> None:
        if self.batch is not None and job.jid in self.batch_ids:
            self.batch.sync()
            self.batch.close()
            self.batch, self.batch_ids = None, ()
        self.samplers.pop(job.jid).close()
        self.means.pop(job.jid)
        self.traces.pop(job.jid, None)
        key, st = self.job_stream.pop(job.jid)
        _STREAMS[key].append(st)


class SlotEngine(GpuEngine):
    """GpuEngine whose FP32 Gaussian jobs live in standing batches of slots
    (``native.Slots``): the launch layout -- block maps and the CUDA graph of
    one batched iteration -- is built once per batch, and admitting or
    retiring a job only edits the slot table on the device.  Slots are
    grouped by capacity into independent batches (by default one per power
    of two from 2^10 to 2^18 particles, ``per_class`` slots each), each with
    its own high-priority stream, so that small jobs do not wait for large
    ones at every stage; every round of a batch advances all its idle jobs
    together (each by its own count) in one launch per stage.  An
    FP32 Gaussian job that fits no free slot waits for one (batched
    iterations are several times cheaper than its own); one larger than
    every slot, FP64 and logistic jobs, and jobs whose statistics are kept
    run one launch per job as in GpuEngine."""

    GROUPS = tuple((c, c) for c in range(10, 19))  # log2 capacity classes per batch: one power of two each

    def __init__(self, device: str = "cuda", per_class: int = 32, groups=GROUPS):
        super().__init__(batched=False, device=device)
        torch = self.torch
        self.groups = []
        for lo, hi in groups:
            caps = [1 << c for c in range(lo, hi + 1) for _ in range(per_class)]
            st = torch.cuda.Stream(device=device, priority=self.hi_prio)
            self.groups.append({"caps": caps, "slots": self.native.Slots(caps, stream=st, device=device),
                                "stream": st, "free": set(range(len(caps))), "busy": False})
        self.slot_of: dict[int, tuple] = {}  # jid -> (group, slot)
        self.max_cap = max(max(g["caps"]) for g in self.groups)

    def _slotted_kind(self, job: Job) -> bool:
        return job.kind == "gauss" and job.dtype == "f32" and not job.keep and job.n <= self.max_cap

    def _try_attach(self, job: Job) -> bool:
        for gi, g in enumerate(self.groups):
            fits = [s for s in g["free"] if g["caps"][s] >= job.n]
            if fits:
                s = min(fits, key=lambda q: (g["caps"][q], q))
                g["free"].discard(s)
                g["slots"].attach(s, self.samplers[job.jid], mean=self.means[job.jid])
                self.slot_of[job.jid] = (gi, s)
                return True
        return False

    def admit(self, job: Job) -> None:
        super().admit(job)
        if self._slotted_kind(job):
            self._try_attach(job)

    def step(self, jobs: list[Job], iters: dict[int, int]) -> list[int]:
        torch = self.torch
        # jobs still waiting for a slot take one that has freed
        for j in jobs:
            if j.jid not in self.slot_of and self._slotted_kind(j):
                self._try_attach(j)
        launched = []
        for gi, g in enumerate(self.groups):
            mine = [j for j in jobs if self.slot_of.get(j.jid, (-1,))[0] == gi]
            if not mine or g["busy"]:
                continue
            counts = [0] * len(g["caps"])
            for j in mine:
                counts[self.slot_of[j.jid][1]] = int(iters[j.jid])
            g["slots"].step(counts)
            ev = torch.cuda.Event()
            ev.record(g["stream"])
            self.pending.append((ev, [j.jid for j in mine], gi))
            g["busy"] = True
            launched += [j.jid for j in mine]
        others = [j for j in jobs if j.jid not in self.slot_of and not self._slotted_kind(j)]
        if others:
            launched += super().step(others, iters)
        return launched

    def completed(self, block: bool = True) -> list[int]:
        if not self.pending:
            return []
        while True:
            done = [p for p in self.pending if p[0].query()]
            if done or not block:
                break
            time.sleep(20e-6)
        self.pending = [p for p in self.pending if p not in done]
        for _, _, tag in done:
            if isinstance(tag, int) and not isinstance(tag, bool):
                self.groups[tag]["busy"] = False
        return [jid for _, ids, _ in done for jid in ids]

    def release(self, job: Job) -> None:
        where = self.slot_of.pop(job.jid, None)
        if where is not None:
            gi, s = where
            self.groups[gi]["slots"].detach(s)
            self.groups[gi]["free"].add(s)
        super().release(job)
