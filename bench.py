"""Benchmark of the SMC-sampler hot path on GB300.

Default workload (one JSON line): one SMC iteration per step -- move, reweight,
LSE/N_eff, estimate, systematic resampling and redistribute (Algorithm 2,
lines 3-10) -- at the resample+redistribute microbenchmark's largest size:
N = 2^24 particles of D = 16 FP32 coordinates, Gaussian target, resampling at
every iteration (the worst case of Sec. 5.2).  value = particle-iterations/s
of the K timed iterations run by one smc_step call (the graph-replayed entry
point a user calls).  A separate pass of smc_step_profile (the same iteration
launched directly, with events between its stages) gives the per-stage times
and the roofline of the dominant kernel.  The line also carries the
stateless resample+redistribute microbenchmark at N = 2^24, D = 16 (the
whole smc_redistribute_raw call and its copy kernel, GB/s against the
measured HBM peak), an end-to-end figure through the C-ABI with host
buffers, and the CPU oracle's rate on a bounded sample.

--workload redistribute prints one line per case of the resample+redistribute
microbenchmark (N in {2^16, 2^20, 2^24}, s in {0.5, 2, 8}, one-hot).
--workload batch: 256 independent FP32 Gaussian-target samplers (N
log-uniform in [2^10, 2^18], D in {2, 8, 32}, resampling when N_eff < N/2),
stepped by one batched launch per stage (CUDA graph, autotuned launch shapes),
against the same samplers stepped one sampler per launch (each its own graph
on its own stream, all streams concurrent; and one after another);
a step is one iteration of every sampler (--steps 50 is the workload's K).
--workload logistic: Bayesian logistic regression, N = 2^18 FP32 particles,
M = 8192 rows, D = 32 features; the likelihood on the tensor cores (tcgen05,
BF16 hi / lo split) next to the CUDA-core FP32 likelihood of the same sampler.
--workload c0: the plain FP64 sampler (N = 1024, D = 4, K = 20, resampling
when N_eff < N/2): time-to-posterior of the K iterations (one CUDA graph
replay each) and the estimate's error against the closed form.
--workload serve: a Poisson stream of sampler jobs (--rate per second, --jobs
jobs): Gaussian jobs of the batched workload (K = 50) mixed with logistic jobs
(N = 2^18, M in {1024, 8192}, D = 32, K = 100; --logistic-frac of the stream),
admitted by free HBM, served with continuous batching; p50 / p99
time-to-posterior and particle-iterations/s, next to the same stream served one
sampler per launch.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
Multi-GPU (torchrun): independent replicas, one sampler per GPU, no collective
on the data path; value = all ranks' particle-iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-iters/s"
STAGES = ["move_reweight", "max_finalize", "quantise_reduce_estimate", "quantise_finalize", "systematic_scan",
          "redistribute", "commit"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="iteration",
                   choices=["iteration", "redistribute", "batch", "logistic", "serve", "c0"])
    p.add_argument("--m", type=int, default=8192, help="logistic workload: data rows")
    p.add_argument("--jobs", type=int, default=2000, help="serve workload: jobs in the Poisson stream")
    p.add_argument("--rate", type=float, default=200.0, help="serve workload: arrivals per second")
    p.add_argument("--logistic-frac", type=float, default=0.1, help="serve workload: share of logistic jobs")
    p.add_argument("--sat-jobs", type=int, default=300, help="serve workload: jobs of the saturated run")
    p.add_argument("--min-batch", type=int, default=16,
                   help="serve workload: fewest ready Gaussian jobs that share a batched launch")
    p.add_argument("--count", type=int, default=256, help="batch workload: samplers")
    p.add_argument("--n", type=int, default=1 << 24)
    p.add_argument("--d", type=int, default=16)
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-redistribute", action="store_true",
                   help="default workload: leave out the redistribute microbenchmark")
    p.add_argument("--sizes", default="16,20,24", help="redistribute workload: log2 N values")
    p.add_argument("--cases", default="s0.5,s2,s8,onehot", help="redistribute workload: weight cases")
    p.add_argument("--seeds", default="0,1,2,3,4", help="redistribute workload: input seeds")
    return p.parse_args()


# ----------------------------------------------------------------- environment
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


STAGE_SOURCES = {
    "move_reweight": ["k_particles.cu", "particle_bodies.cuh", "smc_internal.cuh"],
    "quantise_reduce_estimate": ["k_resample.cu", "particle_bodies.cuh", "smc_internal.cuh"],
    "systematic_scan": ["k_resample.cu", "particle_bodies.cuh", "smc_internal.cuh"],
    "redistribute": ["k_resample.cu", "particle_bodies.cuh", "smc_internal.cuh"],
}


def measured_traffic():
    """DRAM bytes per particle per stage from profiles/traffic.md, kept only
    while the stage's kernel sources are the ones that were captured."""
    import hashlib

    out = {}
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.md")).read().splitlines()
    except OSError:
        return out
    csrc = os.path.join(ROOT, "paper_1905_10252_gb300", "csrc")
    for line in lines:
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) != 7 or cells[0] not in STAGE_SOURCES:
            continue
        h = hashlib.sha256()
        try:
            for f in STAGE_SOURCES[cells[0]]:
                with open(os.path.join(csrc, f), "rb") as fh:
                    h.update(fh.read())
        except OSError:
            continue
        if h.hexdigest()[:16] == cells[2]:
            out[cells[0]] = float(cells[6])
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples with host timestamps."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [p for (t, p) in self.samples if t0 <= t <= t1]
        note = "samples inside the timed region"
        if not inside and self.samples:
            # timed region shorter than the sampling period: nearest samples
            mid = 0.5 * (t0 + t1)
            inside = [min(self.samples, key=lambda s: abs(s[0] - mid))[1]]
            note = "nearest sample (timed region shorter than the 100 ms sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        sm = [float(p[1]) for p in inside if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in inside if p[2].replace(".", "").isdigit()]
        reasons = sorted({names[j] for p in inside for j in range(4) if p[4 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "note": note}


# ----------------------------------------------------------------- CPU baseline (oracle)
def oracle_iteration_rate(n_sample: int, iters: int, d: int, seed: int = 0):
    """The FP64 oracle's Algorithm 2 iteration (move, reweight, LSE/N_eff,
    estimate, resample, redistribute, reset) on n_sample particles."""
    from oracle import oracle as O
    from paper_1905_10252_gb300 import inputs

    mu, Sigma = inputs.gaussian_target(d, seed=16)
    tgt = O.Target.gauss(mu, Sigma)
    x, lw, lp = O.init(tgt, n_sample, seed, 2.0, ubits=24)
    t0 = time.perf_counter()
    for t in range(1, iters + 1):
        x1 = O.move(x, seed, t, 0.5, ubits=24)
        lw, lp = O.reweight(tgt, x, x1, lp, lw, 0.5)
        m, lse, ess = O.lse_ess(lw)
        O.estimate(x1, lw, lse, with_cov=False)
        r = O.resample(lw, seed, t, O.RESAMPLE_ALWAYS)
        x = O.redistribute(r["ncopies"], x1)
        lp = O.redistribute(r["ncopies"], lp)
        lw = np.full(n_sample, O.reset_logw(n_sample))
    dt = time.perf_counter() - t0
    return n_sample * iters / dt, dt


def cpu_baseline(d: int):
    n_sample, iters = 1 << 20, 20
    rate, dt = oracle_iteration_rate(n_sample, iters, d)
    return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{iters} iterations of N={n_sample} (D={d}, FP64, single thread), {dt:.1f} s",
            "host_cpus": os.cpu_count()}


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    d = args.d
    # each step is one oracle iteration on a sample sized so that warmup+steps
    # take about a minute in all
    per = 1.6e-6
    n_sample = int(max(1024, min(1 << 18, 60.0 / max(1, args.steps + args.warmup) / per)))
    from oracle import oracle as O
    from paper_1905_10252_gb300 import inputs

    mu, Sigma = inputs.gaussian_target(d, seed=16)
    tgt = O.Target.gauss(mu, Sigma)
    x, lw, lp = O.init(tgt, n_sample, 0, 2.0, ubits=24)
    times = []
    for t in range(1, args.warmup + args.steps + 1):
        t0 = time.perf_counter()
        x1 = O.move(x, 0, t, 0.5, ubits=24)
        lw, lp = O.reweight(tgt, x, x1, lp, lw, 0.5)
        m, lse, ess = O.lse_ess(lw)
        O.estimate(x1, lw, lse, with_cov=False)
        r = O.resample(lw, 0, t, O.RESAMPLE_ALWAYS)
        x = O.redistribute(r["ncopies"], x1)
        lp = O.redistribute(r["ncopies"], lp)
        lw = np.full(n_sample, O.reset_logw(n_sample))
        if t > args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_sample * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"smc-iteration gauss N=2^24 (sampled: N={n_sample}) D={d} resample-every-iteration"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"N={n_sample} particles per step, FP64 oracle, single thread"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
def max_over_ranks(local_ms: float, world_size: int, device="cpu") -> float:
    """The step time of the whole job: the slowest rank's (replicas of the
    sampler run independently; this is the only collective, outside the
    timed region)."""
    if world_size <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, steps: int, world_size: int, total_ms: float) -> float:
    """Whole-job particle-iterations per second (weak scaling: every rank runs
    its own N-particle sampler)."""
    return n_per_rank * steps * world_size / (total_ms * 1e-3)


def algorithmic_bytes(n: int, d: int, esize: int, survivors: float, est_in_move: bool = False,
                      gather: bool = False):
    """Per-launch algorithmic bytes of each stage (see the measurement section
    of the design notes): reads + writes the definition of the stage needs.
    est_in_move: the move kernel formed the sums of eq. (7) (FP32 Gaussian,
    D <= 16, every log w equal after the previous resampling), so the
    quantise pass reads log w only.  gather: the previous iteration's
    redistribution is done by this move (the rows of the survivors read once
    through the run starts, every log w equal to -log N), and there is no
    copy stage."""
    row = d * esize
    if gather:
        return {
            # read the run starts, the distinct surviving rows + log pi; write
            # x, log pi, log w
            "move_reweight": n * 4 + survivors * (row + esize) + n * (row + esize + 8),
            "quantise_reduce_estimate": n * 8,
            "systematic_scan": n * 8 + survivors * 4,
        }
    return {
        # read x, log pi, log w; write x, log pi, log w
        "move_reweight": n * (2 * row + 2 * esize + 2 * 8),
        # read log w (quantisation) and x (the weighted mean of eq. (7)),
        # unless the move kernel formed the mean
        "quantise_reduce_estimate": n * 8 if est_in_move else n * (8 + row),
        # read log w, write one run start per survivor (the ncopies information)
        "systematic_scan": n * 8 + survivors * 4,
        # read the run starts, the distinct surviving rows + log pi, write
        # N rows + log pi, reset N log-weights
        "redistribute": n * 4 + survivors * (row + esize) + n * (row + esize) + n * 8,
    }


def time_redistribute(native, torch, nc, x, out, wsb, flush, warmup: int, reps: int):
    """(call ms, copy-kernel ms) of smc_redistribute_raw_profile per timed
    repetition, L2 flushed before each: the whole stateless call (its ncopies
    scan, then the copy) and the copy kernel alone."""
    res = []
    for it in range(warmup + reps):
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        native.smc_redistribute_raw_profile(nc, x, out, wsb, evs)
        torch.cuda.synchronize()
        if it >= warmup:
            res.append((evs[0].elapsed_time(evs[2]), evs[1].elapsed_time(evs[2])))
    return res


def redistribute_summary(n: int, d: int, cases, seed: int, reps: int, peak: float):
    """The resample+redistribute microbenchmark at one size for the default
    line: per weight case, medians of the stateless call and of its copy
    kernel; bytes = run starts / ncopies 4 + distinct source rows 64 rho +
    written rows 64, per row."""
    import torch

    from paper_1905_10252_gb300 import inputs, native

    x = torch.as_tensor(inputs.particles(n, d, seed=1), device="cuda")
    out = torch.empty_like(x)
    wsb = torch.empty(native.smc_redistribute_ws_bytes(n), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    row = d * 4
    per_case = {}
    for case in cases:
        lw = inputs.one_hot_log_weights(n, seed) if case == "onehot" else inputs.log_weights(n, float(case[1:]), seed)
        native.smc_resample_raw(torch.as_tensor(lw, device="cuda"), seed, 1, native.RESAMPLE_ALWAYS, ncopies=nc,
                                ws=wsb)
        nnz = int((nc > 0).sum().item())
        byt = 4 * n + row * nnz + row * n
        t = time_redistribute(native, torch, nc, x, out, wsb, flush, 3, reps)
        call_ms = statistics.median(c for c, _ in t)
        copy_ms = statistics.median(k for _, k in t)
        per_case[case] = {"survivors": nnz, "bytes": byt,
                          "call_ms": round(call_ms, 5), "call_gbs": round(byt / (call_ms * 1e-3) / 1e9, 1),
                          "call_frac": round(byt / (call_ms * 1e-3) / 1e9 / peak, 4),
                          "copy_ms": round(copy_ms, 5), "copy_gbs": round(byt / (copy_ms * 1e-3) / 1e9, 1),
                          "copy_frac": round(byt / (copy_ms * 1e-3) / 1e9 / peak, 4)}
    del x, out, wsb, flush, nc
    torch.cuda.empty_cache()
    return {"workload": f"stateless resample+redistribute N=2^{int(np.log2(n))} D={d} fp32 rows, seed {seed}",
            "entry_point": "smc_redistribute_raw (ncopies scan + copy); copy = its copy kernel alone",
            "bytes": "4 + 64 rho + 64 per row (rho = survivors / N)", "unit": "GB/s", "peak": peak,
            "timing": f"median of {reps} calls per case, L2 flushed before each", "cases": per_case,
            "min_call_frac": min(c["call_frac"] for c in per_case.values()),
            "min_copy_frac": min(c["copy_frac"] for c in per_case.values())}


def run_iteration(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300 import inputs, native

    n, d = args.n, args.d
    mu, Sigma = inputs.gaussian_target(d, seed=16)
    # (D <= 16: each resampling's copy is gathered by the next iteration's
    # move; the particles and weights are those of the copying iteration)
    gather = d <= 16
    S = native.Sampler(n, d, dtype=torch.float32, seed=rank, mu=mu, sigma=Sigma, step=0.5, init_scale=2.0,
                       resample_mode=native.RESAMPLE_ALWAYS,
                       flags=native.FLAG_DEFER_REDISTRIBUTE if gather else 0)
    stream = S.stream
    K, W = args.steps, args.warmup
    L = native.lib()
    mean_d = torch.empty(d, dtype=torch.float64, device="cuda")

    def product_step(k):
        # the entry point a user calls: k iterations replayed from the
        # sampler's CUDA graph, f_k into mean_d
        S._enter()
        native._check(L.smc_step(S.h, int(k), native._ptr(mean_d), None, None, None), S.h)
        S._done()

    for _ in range(W):
        product_step(1)
    torch.cuda.synchronize()
    n_prof = max(5, min(K, 50))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_prof)]
    for row in ev:
        for e in row:
            e.record(stream)  # creates the event
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.time()
    start.record(stream)
    product_step(K)
    stop.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    if ws > 1:
        dist.barrier()
    # per-stage split: the same iteration launched directly with events
    # between its stages (smc_step_profile), run right after the timed region
    # on the same sampler (every one of these iterations resamples too)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(n_prof):
        S.step_profile(ev[k])
    p1.record(stream)
    torch.cuda.synchronize()
    t_host2 = time.time()
    time.sleep(0.15)
    clocks.stop()
    total_ms = max_over_ranks(start.elapsed_time(stop), ws, device="cuda")
    prof_ms_per_iter = p0.elapsed_time(p1) / n_prof
    per_stage = {name: [] for name in STAGES}
    for row in ev:
        for j, name in enumerate(STAGES):
            per_stage[name].append(row[j].elapsed_time(row[j + 1]))
    stage_ms = {k: float(np.mean(v)) for k, v in per_stage.items()}
    st = S.stats()
    survivors = float(st["survivors"])
    # every timed iteration resamples, so each one starts from equal weights
    byt = algorithmic_bytes(n, d, 4, survivors, est_in_move=d <= 16, gather=gather)
    peak, peak_kind = peaks()
    dominant = max(stage_ms, key=stage_ms.get)
    traffic = measured_traffic()

    def roof(name):
        if name not in byt:
            return None
        gbs = byt[name] / (stage_ms[name] * 1e-3) / 1e9
        tr = int(traffic[name] * n) if name in traffic else None
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4), "traffic": tr, "peak_kind": peak_kind,
                "bytes_per_launch": int(byt[name]), "ms_per_launch": round(stage_ms[name], 5)}

    # end to end through the public API with host buffers: pinned H2D of the
    # particle state, one iteration, D2H of the estimate and its statistics
    e2e = None
    if args.e2e_steps > 0:
        x_h = S.current()[0].cpu().pin_memory()
        lp_h = S.current()[1].cpu().pin_memory()
        lw_h = S.logw.cpu().pin_memory()
        # (samplers that copy at the end of each iteration: every step here
        # replaces the whole state from the host buffers)
        S.close()
        S = native.Sampler(n, d, dtype=torch.float32, seed=rank, mu=mu, sigma=Sigma, step=0.5, init_scale=2.0,
                           resample_mode=native.RESAMPLE_ALWAYS)
        stream = S.stream
        mean_d = torch.empty(d, dtype=torch.float64, device="cuda")
        mean_h = torch.empty(d, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = S.current()
        which = 0 if cur[0].data_ptr() == S.x.data_ptr() else 1
        e0.record(stream)
        for _ in range(args.e2e_steps):
            xs, lps = (S.x, S.logpi) if which == 0 else (S.x_alt, S.logpi_alt)
            with torch.cuda.stream(stream):
                xs.copy_(x_h, non_blocking=True)
                lps.copy_(lp_h, non_blocking=True)
                S.logw.copy_(lw_h, non_blocking=True)
            S.step_profile(mean=mean_d)
            with torch.cuda.stream(stream):
                mean_h.copy_(mean_d, non_blocking=True)
            which ^= 1  # resampling at every iteration swaps the buffers
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        serial = {"value": n * args.e2e_steps / (e_ms * 1e-3), "ms_per_step": e_ms / args.e2e_steps}
        # pipelined: steps alternate between S and a second sampler of the same
        # configuration; each step's host copies run on its sampler's copy
        # stream as soon as that sampler's previous step is done with its
        # buffers, so they overlap the other sampler's iteration (the host link,
        # not the GPU, bounds this measurement)
        L = native.lib()
        S2 = native.Sampler(n, d, dtype=torch.float32, seed=rank + 7, mu=mu, sigma=Sigma, step=0.5,
                            init_scale=2.0, resample_mode=native.RESAMPLE_ALWAYS)
        pair = [S, S2]
        cur_idx = [0 if T.current()[0].data_ptr() == T.x.data_ptr() else 1 for T in pair]
        copy_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        free_ev = [torch.cuda.Event(), torch.cuda.Event()]
        means_d = [torch.empty(d, dtype=torch.float64, device="cuda") for _ in pair]
        means_h = [torch.empty(d, dtype=torch.float64).pin_memory() for _ in pair]
        master = torch.cuda.current_stream()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(master)
        for j in range(2):
            free_ev[j].record(master)
        for k in range(args.e2e_steps):
            j = k & 1
            T, cs = pair[j], copy_streams[j]
            cs.wait_event(free_ev[j])
            xs, lps = (T.x, T.logpi) if cur_idx[j] == 0 else (T.x_alt, T.logpi_alt)
            with torch.cuda.stream(cs):
                xs.copy_(x_h, non_blocking=True)
                lps.copy_(lp_h, non_blocking=True)
                T.logw.copy_(lw_h, non_blocking=True)
            T.stream.wait_stream(cs)
            native._check(L.smc_step_profile(T.h, native._ptr(means_d[j]), None, 0), T.h)
            with torch.cuda.stream(T.stream):
                means_h[j].copy_(means_d[j], non_blocking=True)
            free_ev[j].record(T.stream)
            cur_idx[j] ^= 1
        for T in pair:
            master.wait_stream(T.stream)
        p1.record(master)
        torch.cuda.synchronize()
        S2.sync()
        p_ms = p0.elapsed_time(p1)
        S2.close()
        e2e = {"value": n * args.e2e_steps / (p_ms * 1e-3), "unit": METRIC,
               "h2d_bytes_per_step": int(x_h.nbytes + lp_h.nbytes + lw_h.nbytes),
               "d2h_bytes_per_step": int(mean_h.nbytes), "ms_per_step": p_ms / args.e2e_steps,
               "mode": "two samplers alternate; each step's host copies overlap the other's iteration",
               "serial": serial}
    S.sync()
    value = job_value(n, K, ws, total_ms)
    # the stateless resample+redistribute microbenchmark at N = 2^24, D = 16
    # (the metric's redistribute GB/s), rank 0 of a single-GPU run
    redist = None
    if rank == 0 and ws == 1 and not args.no_redistribute:
        redist = redistribute_summary(1 << 24, 16, ["s0.5", "s2", "s8", "onehot"], 0, 20, peak)
    # one step set-up per smc_step call, then per iteration: begin, move +
    # reweight, max, quantise reduce / finalise, scan, (redistribute,) commit
    launches_per_step = 7 if gather else 8
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state / f64 weights / u64 fixed-point CDF", "data": "synthetic",
            "config": {"workload": f"smc-iteration gauss N=2^{int(np.log2(n))} D={d} fp32 resample-every-iteration",
                       "n": n, "d": d, "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (particle state %.2f GB per buffer)" % (n * d * 4 / 1e9),
                       "redistribute": ("gathered by the next iteration's move (SMC_FLAG_DEFER_REDISTRIBUTE)"
                                        if gather else "copy kernel at the end of the iteration")},
            "entry_point": f"smc_step (one call, {K} iterations replayed from the sampler's CUDA graph)",
            "roofline": roof(dominant) if dominant in byt else roof("move_reweight"),
            "dominant_kernel": dominant,
            "profile_pass": {"entry_point": "smc_step_profile (direct launches, events between stages)",
                             "iterations": n_prof, "ms_per_iteration": round(prof_ms_per_iter, 5),
                             "ratio_to_timed": round(prof_ms_per_iter / (total_ms / K), 4),
                             "note": "stage times, stage_roofline and roofline come from this pass"},
            "redistribute": redist,
            "stages_ms": {k: round(v, 5) for k, v in stage_ms.items()},
            "stage_roofline": {k: roof(k) for k in byt},
            "survivors_last_iteration": int(survivors),
            "gpu_launches": 1 + launches_per_step * K,
            "clocks": clocks.summary(t_host0, t_host1),
            "clocks_profile_pass": clocks.summary(t_host1, t_host2),
            "e2e": e2e,
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(d)
        print(json.dumps(line), flush=True)
    S.close()
    if ws > 1:
        dist.destroy_process_group()


def run_redistribute(args):
    """Resample + redistribute microbenchmark: i.i.d. N(0, s^2) log-weights or
    one-hot; resampling then redistribute of D=16 FP32 rows."""
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300 import inputs, native

    peak, peak_kind = peaks()
    d = args.d
    for n in [1 << int(v) for v in args.sizes.split(",")]:
        x = torch.as_tensor(inputs.particles(n, d, seed=1), device="cuda")
        out = torch.empty_like(x)
        wsb = torch.empty(native.smc_redistribute_ws_bytes(n), dtype=torch.uint8, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        # the paper's N-R local step for comparison: S-NS (Algorithm 8), then
        # S-R on the nearly-sorted keys and rows
        ns_keys, ns_rows, nr_out = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty_like(x),
                                    torch.empty_like(x))
        wsn = torch.empty(native.smc_nearly_sort_ws_bytes(n), dtype=torch.uint8, device="cuda")
        row_bytes = d * 4
        seeds = [int(v) for v in args.seeds.split(",")]
        for case in args.cases.split(","):
            nc = torch.empty(n, dtype=torch.int32, device="cuda")
            # per timed iteration: (ms, algorithmic bytes) of each measured part
            res, red, cop, nsr, nr = [], [], [], [], []
            survivors = []
            for seed in seeds:
                lw = (inputs.one_hot_log_weights(n, seed) if case == "onehot"
                      else inputs.log_weights(n, float(case[1:]), seed))
                lwd = torch.as_tensor(lw, device="cuda")
                for it in range(args.warmup + 20):
                    flush.zero_()  # L2 flush between iterations
                    a, b, c = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    a.record()
                    native.smc_resample_raw(lwd, seed, it + 1, native.RESAMPLE_ALWAYS, ncopies=nc, ws=wsb)
                    b.record()
                    flush.zero_()
                    b2 = torch.cuda.Event(enable_timing=True)
                    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    b2.record()
                    native.smc_redistribute_raw_profile(nc, x, out, wsb, evs)
                    c.record()
                    flush.zero_()
                    e0, e1, e2 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    e0.record()
                    native.smc_nearly_sort_raw(nc, x, ns_keys, ns_rows, ws=wsn)
                    e1.record()
                    native.smc_redistribute_raw(ns_keys, ns_rows, nr_out, ws=wsb)
                    e2.record()
                    torch.cuda.synchronize()
                    if it >= args.warmup:
                        nnz = int((nc > 0).sum().item())
                        survivors.append(nnz)
                        res.append((a.elapsed_time(b), 8 * n + 8 * n + 4 * n))
                        red.append((b2.elapsed_time(c), 4 * n + row_bytes * nnz + row_bytes * n))
                        # the copy kernel alone: run starts 4 B per row, distinct source rows, N rows written
                        cop.append((evs[1].elapsed_time(evs[2]), 4 * n + row_bytes * nnz + row_bytes * n))
                        nsr.append((e0.elapsed_time(e1), 8 * n + 2 * row_bytes * n))
                        nr.append((e0.elapsed_time(e2), 0))

            def med_ms(v):
                return statistics.median(t for t, _ in v)

            def med_gbs(v):
                return statistics.median(byt / (t * 1e-3) / 1e9 for t, byt in v)

            rm, dm, cm, sm_, nm = med_ms(res), med_ms(red), med_ms(cop), med_ms(nsr), med_ms(nr)
            line = {"metric": "redistribute GB/s", "workload": f"resample+redistribute N=2^{int(np.log2(n))} {case}",
                    "n": n, "d": d, "seeds": seeds, "survivors_median": int(statistics.median(survivors)),
                    "resample_ms": rm, "redistribute_ms": dm,
                    "redistribute_gbs": med_gbs(red), "resample_gbs": med_gbs(res),
                    "peak_gbs": peak, "peak_kind": peak_kind,
                    "redistribute_frac": med_gbs(red) / peak,
                    "copy_kernel_ms": cm, "copy_kernel_gbs": med_gbs(cop), "copy_kernel_frac": med_gbs(cop) / peak,
                    "nearly_sort_ms": sm_, "nearly_sort_gbs": med_gbs(nsr), "nearly_sort_frac": med_gbs(nsr) / peak,
                    "nr_ms": nm, "nr_over_gather": nm / dm,
                    "timing": f"medians over {len(seeds)} seeds x 20 iterations (after {args.warmup} warm-up "
                              "iterations per seed), L2 flushed"}
            if rank == 0:
                print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched samplers against one sampler per launch on the same GPU."""
    import ctypes as C

    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300 import inputs, native

    shapes = inputs.batch_shapes(args.count, seed=0)
    mem = []
    for j, (n, d) in enumerate(shapes):
        mu, sig = inputs.gaussian_target(d, seed=1000 + j)
        mem.append(native.Sampler(n, d, dtype=torch.float32, seed=rank * 100000 + j, mu=mu, sigma=sig, step=0.5,
                                  init_scale=2.0, resample_mode=native.RESAMPLE_ESS))
    total_n = sum(n for n, _ in shapes)
    K, W = args.steps, args.warmup
    L = native.lib()
    master = torch.cuda.Stream()
    torch.cuda.synchronize()

    def solo(concurrent: bool, k: int) -> float:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(master)
        prev = master
        for m in mem:
            m.stream.wait_stream(master if concurrent else prev)
            native._check(L.smc_step(m.h, int(k), None, None, None, None), m.h)
            prev = m.stream
        for m in mem:
            master.wait_stream(m.stream)
        e1.record(master)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    solo(True, W)
    solo_conc_ms = solo(True, K)
    solo_ser_ms = solo(False, K)

    bt = native.Batch(mem)
    t0 = time.time()
    choice = bt.tune(reps=5)
    tune_s = time.time() - t0
    bt.step_raw(W)
    n_prof = 20
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_prof)]
    for row in ev:
        for e in row:
            e.record(bt.stream)  # creates the event
    for row in ev:
        bt.step_profile(row)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    start.record(bt.stream)
    bt.step_raw(K)
    stop.record(bt.stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    time.sleep(0.15)
    clocks.stop()
    bt.sync()
    batch_ms = max_over_ranks(start.elapsed_time(stop), ws, device="cuda")
    stage_ms = {name: float(np.mean([row[j].elapsed_time(row[j + 1]) for row in ev]))
                for j, name in enumerate(STAGES)}
    # algorithmic bytes of the stages that do not depend on the resampling decision
    mv_bytes = sum(n * (2 * 4 * d + 2 * 4 + 2 * 8) for n, d in shapes)
    # (rows counted for every member: an upper bound, since members with
    # D <= 16 read log w only in iterations that follow a resampling)
    q_bytes = sum(n * (8 + 4 * d) for n, d in shapes)
    peak, peak_kind = peaks()

    def roof(name, byt):
        gbs = byt / (stage_ms[name] * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                "traffic": None, "peak_kind": peak_kind, "bytes_per_launch": int(byt),
                "ms_per_launch": round(stage_ms[name], 5)}

    value = job_value(total_n, K, ws, batch_ms)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": batch_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state / f64 weights / u64 fixed-point CDF", "data": "synthetic",
            "config": {"workload": f"batched {args.count} gauss samplers N log-uniform [2^10,2^18] D in {{2,8,32}} "
                                   "fp32 resample when N_eff < N/2",
                       "samplers": args.count, "total_particles": total_n, "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (state %.2f GB)" % (sum(n * d * 4 * 2 for n, d in shapes) / 1e9)},
            "one_sampler_per_launch": {
                "concurrent_streams": {"value": job_value(total_n, K, ws, solo_conc_ms), "ms_per_step": solo_conc_ms / K},
                "one_after_another": {"value": job_value(total_n, K, ws, solo_ser_ms), "ms_per_step": solo_ser_ms / K}},
            "speedup_vs_concurrent_solo": solo_conc_ms / batch_ms,
            "tuned_variant": {"move": choice[0], "copy": choice[1], "tune_s": round(tune_s, 3)},
            "roofline": roof("move_reweight", mv_bytes),
            "dominant_kernel": max(stage_ms, key=stage_ms.get),
            "stage_roofline": {"move_reweight": roof("move_reweight", mv_bytes),
                               "quantise_reduce_estimate": roof("quantise_reduce_estimate", q_bytes)},
            "stages_ms": {k: round(v, 5) for k, v in stage_ms.items()},
            "gpu_launches": 8 * K,
            "clocks": clocks.summary(t_host0, t_host1),
        }
        print(json.dumps(line), flush=True)
    bt.close()
    for m in mem:
        m.close()


def run_logistic(args):
    """Bayesian logistic regression sampler: tensor-core likelihood."""
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300 import inputs, native

    n, d, m = (args.n if args.n != (1 << 24) else 1 << 18), 32, args.m
    X, y, _ = inputs.logistic_data(m, d, seed=0)

    def sampler(flags):
        # q_0 = the prior N(0, 4I), random-walk step 0.5 (the configuration's
        # reading; the posterior estimate itself is poor without tempering)
        return native.Sampler(n, d, dtype=torch.float32, seed=rank, target="logistic", X=X, y=y, prior_var=4.0,
                              step=0.5, init_scale=2.0, flags=flags)

    S = sampler(0)
    K, W = args.steps, args.warmup
    for _ in range(W):
        S.step_profile()
    n_prof = 10
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(n_prof)]
    for row in ev:
        for e in row:
            e.record(S.stream)
    for row in ev:
        S.step_profile(row)
    torch.cuda.synchronize()
    stage_ms = {name: float(np.mean([row[j].elapsed_time(row[j + 1]) for row in ev])) for j, name in enumerate(STAGES)}
    clocks = ClockSampler(local)
    time.sleep(0.3)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_host0 = time.time()
    start.record(S.stream)
    S.step(K)
    stop.record(S.stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    time.sleep(0.15)
    clocks.stop()
    S.sync()
    total_ms = max_over_ranks(start.elapsed_time(stop), ws, device="cuda")
    # the CUDA-core FP32 likelihood on the same workload (a few iterations)
    C = sampler(native.FLAG_LOGISTIC_CUDA_CORES)
    cev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(3)]
    for row in cev:
        for e in row:
            e.record(C.stream)
    C.step_profile()
    for row in cev:
        C.step_profile(row)
    torch.cuda.synchronize()
    cc_ms = float(np.mean([row[0].elapsed_time(row[1]) for row in cev]))
    C.close()
    clk = clocks.summary(t_host0, t_host1)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    lik_ms = stage_ms["move_reweight"]
    elems = float(n) * float(((m + 255) // 256) * 256)
    mufu_peak = 152 * 16 * sm_mhz * 1e6 / 1.0625  # elements/s: one ex2 + 1/16 lg2 per element, 16 MUFU lanes / SM
    tensor_flops = 3 * 2.0 * elems * 32
    meas = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            meas = json.load(f)
    except OSError:
        pass
    bf16_peak = float(meas.get("bf16_tflops", 1900.0))
    value = job_value(n, K, ws, total_ms)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state / bf16x3 tensor contraction, f32 accumulate / f64 weights", "data": "synthetic",
            "config": {"workload": f"logistic regression N=2^{int(np.log2(n))} M={m} D={d} fp32 resample when "
                                   "N_eff < N/2", "n": n, "m": m, "d": d, "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "alu", "achieved": round(elems / (lik_ms * 1e-3) / 1e9, 1),
                         "peak": round(mufu_peak / 1e9, 1), "unit": "Gelem/s",
                         "frac": round(elems / (lik_ms * 1e-3) / mufu_peak, 4), "traffic": None,
                         "note": "move + likelihood stage; peak = MUFU rate at the sampled SM clock / 1.0625 ops "
                                 "per element"},
            "tensor": {"achieved_tflops": round(tensor_flops / (lik_ms * 1e-3) / 1e12, 1),
                       "peak_tflops": bf16_peak, "frac": round(tensor_flops / (lik_ms * 1e-3) / 1e12 / bf16_peak, 4)},
            "likelihood_ms": {"tensor_cores": round(lik_ms, 4), "cuda_cores_fp32": round(cc_ms, 4),
                              "speedup": round(cc_ms / lik_ms, 2)},
            "stages_ms": {k: round(v, 5) for k, v in stage_ms.items()},
            "gpu_launches": 9 * K,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    S.close()


def serve_jobs(count: int, rate: float, logistic_frac: float, seed: int = 0):
    from paper_1905_10252_gb300 import inputs
    from paper_1905_10252_gb300.serve import Job, poisson_arrivals

    arr = poisson_arrivals(count, rate, seed=seed)
    g = np.random.default_rng(seed + 1)
    kinds = g.uniform(size=count) < logistic_frac
    shapes = inputs.batch_shapes(count, seed=seed + 2)
    datasets = {m: inputs.logistic_data(m, 32, seed=m)[:2] for m in (1024, 8192)}
    targets = {}
    jobs = []
    for i in range(count):
        if kinds[i]:
            m = 1024 if g.uniform() < 0.5 else 8192
            X, y = datasets[m]
            jobs.append(Job(jid=i, kind="logistic", n=1 << 18, d=32, k=100, seed=i, arrival=float(arr[i]), X=X, y=y,
                            step=0.5, init_scale=2.0))
        else:
            n, d = shapes[i]
            if (d, i % 8) not in targets:
                targets[(d, i % 8)] = inputs.gaussian_target(d, seed=1000 + 8 * d + i % 8)
            mu, sig = targets[(d, i % 8)]
            jobs.append(Job(jid=i, kind="gauss", n=n, d=d, k=50, seed=i, arrival=float(arr[i]), mu=mu, sigma=sig))
    return jobs


def run_serve(args):
    """Continuous-batching server on a Poisson stream of jobs: the standing
    batch of slots (the served engine), the batch rebuilt per membership
    change, and one sampler per launch, on the same stream of jobs."""
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300.serve import GpuEngine, Scheduler, SlotEngine, latency_summary

    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.6, 64 << 30))
    engines = {
        "slots": lambda: SlotEngine(),
        "batch_rebuilt_per_change": lambda: GpuEngine(batched=True, min_batch=args.min_batch),
        "one_sampler_per_launch": lambda: GpuEngine(batched=False),
    }
    out = {}
    # warm-up: a short stream through every engine (kernels, allocator, graphs)
    for make in engines.values():
        Scheduler(make(), budget_bytes=budget).run(serve_jobs(40, 400.0, args.logistic_frac, 99))
    for name, make in engines.items():
        jobs = serve_jobs(args.jobs, args.rate, args.logistic_frac, seed=rank)
        eng = make()
        sch = Scheduler(eng, budget_bytes=budget, round_iters=5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = sch.run(jobs, t0=t0)
        wall = time.perf_counter() - t0
        pits = sum(j.n * j.k for j in done)
        gauss = [j for j in done if j.kind == "gauss"]
        logi = [j for j in done if j.kind != "gauss"]
        out[name] = dict(latency_summary(done), wall_s=round(wall, 3), particle_iters_per_s=pits / wall,
                         rounds=sch.rounds, jobs_per_s=len(done) / wall,
                         gauss=latency_summary(gauss) if gauss else None,
                         logistic=latency_summary(logi) if logi else None)
    # saturation: every job waiting at t = 0 (throughput), the mix and the
    # Gaussian jobs alone
    for tag, frac in (("saturated", args.logistic_frac), ("saturated_gauss_only", 0.0)):
        sat = {}
        for name in ("slots", "one_sampler_per_launch"):
            jobs = serve_jobs(args.sat_jobs, args.rate, frac, seed=rank + 7)
            for j in jobs:
                j.arrival = 0.0
            sch = Scheduler(engines[name](), budget_bytes=budget, round_iters=5)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            done = sch.run(jobs, t0=t0)
            wall = time.perf_counter() - t0
            sat[name] = {"jobs": len(done), "wall_s": round(wall, 3),
                         "particle_iters_per_s": sum(j.n * j.k for j in done) / wall, "rounds": sch.rounds}
        sat["speedup"] = sat["slots"]["particle_iters_per_s"] / sat["one_sampler_per_launch"]["particle_iters_per_s"]
        out[tag] = sat
    b = out["slots"]
    if rank == 0:
        line = {
            "metric": "served p50/p99 time-to-posterior; particle-iters/s", "value": b["particle_iters_per_s"],
            "unit": METRIC, "n_gpus": ws, "steps": args.jobs, "warmup": 40, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 state / f64 weights", "data": "synthetic",
            "config": {"workload": f"serve Poisson {args.rate:g} jobs/s x {args.jobs}: gauss (batched workload, "
                                   f"K=50) + {args.logistic_frac:.0%} logistic (N=2^18, M in {{1024,8192}}, D=32, "
                                   "K=100)", "budget_bytes": budget, "round_iters": 5,
                       "engine": "standing batches of slots (one per capacity class 2^10..2^18, 32 slots each)",
                       "parallelism": f"replicas x{ws}"},
            "p50_s": b["p50_s"], "p99_s": b["p99_s"],
            "serving": out,
            "p99_vs_one_sampler_per_launch": b["p99_s"] / out["one_sampler_per_launch"]["p99_s"],
            "saturated_speedup_vs_one_sampler_per_launch": out["saturated"]["speedup"],
            "saturated_gauss_only_speedup_vs_one_sampler_per_launch": out["saturated_gauss_only"]["speedup"],
        }
        print(json.dumps(line), flush=True)


def run_c0(args):
    """Plain FP64 sampler, N = 1024, D = 4, K = 20: time-to-posterior."""
    import torch

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1905_10252_gb300 import build as B

    B.build()
    from paper_1905_10252_gb300 import inputs, native

    N, D, K = 1024, 4, 20
    mu, Sigma = inputs.gaussian_target(D, seed=0)
    reps = max(args.steps, 1)
    times, cold, errs = [], [], []
    for r in range(args.warmup + reps):
        # cold: a fresh sampler's first K iterations; warm: K more iterations
        # of the same sampler (the steady cost of a resident job).  smc_step
        # runs the K iterations of this FP64 sampler of 1024 particles in one
        # cooperative launch (then the covariance and the last copy)
        S = native.Sampler(N, D, dtype=torch.float64, seed=r, mu=mu, sigma=Sigma, step=0.5, init_scale=2.0)
        torch.cuda.synchronize()
        e0, e1, e2 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e0.record(S.stream)
        out = S.step(K, cov=True)
        e1.record(S.stream)
        S.step(K, cov=True)
        e2.record(S.stream)
        torch.cuda.synchronize()
        if r >= args.warmup:
            cold.append(e0.elapsed_time(e1) * 1e3)
            times.append(e1.elapsed_time(e2) * 1e3)
            errs.append(np.abs(out["mean"].cpu().numpy() - mu).max())
        S.close()
    us = float(np.median(times))
    if rank == 0:
        print(json.dumps({
            "metric": "time-to-posterior", "value": us, "unit": "us", "n_gpus": ws, "steps": reps, "warmup": args.warmup,
            "ms_per_step": us / 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "plain fp64 sampler N=1024 D=4 K=20 gauss, resample when N_eff < N/2",
                       "timing": f"median over {reps} runs (seeds) of K more iterations of a resident sampler "
                                 "(one smc_step call), CUDA events on its stream",
                       "entry_point": "smc_step (K iterations in one cooperative launch, then the covariance "
                                      "and the last copy + commit)"},
            "particle_iters_per_s": N * K / (us * 1e-6), "cold_us_first_call": float(np.median(cold)),
            "mean_abs_err_max_vs_closed_form": {"median": float(np.median(errs)), "max": float(np.max(errs))},
            "gpu_launches": 5}), flush=True)  # step set-up, the fused iterations, covariance (2), copy + commit


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "redistribute":
        run_redistribute(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "logistic":
        run_logistic(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "c0":
        run_c0(args)
    else:
        run_iteration(args)


if __name__ == "__main__":
    main()
