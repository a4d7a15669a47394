"""Deferred redistribution (SMC_FLAG_DEFER_REDISTRIBUTE): Algorithm 5 done as a
gather inside the next iteration's move instead of a copy at the end of the
resampling iteration.  The move and reweight of particle k depend only on k
and on the row it starts from, so every particle, log pi, log w, estimate and
statistic must be bit-identical to those of the sampler without the flag:
over whole runs in one smc_step call, across calls (the redistribution
pending in between), with N_eff-based decisions (some iterations keep their
weights), in heavily duplicated resamplings (long runs of copies, whose
sources come from the copy-tile starts), and when another call completes a
pending redistribution first."""
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


def _pair(nat, N, D, mode, seed=3, step=0.5, mu=None, sigma=None):
    if mu is None:
        mu, sigma = inputs.gaussian_target(D, seed=D)
    kw = dict(dtype=torch.float32, seed=seed, mu=mu, sigma=sigma, step=step, resample_mode=mode)
    return nat.Sampler(N, D, **kw), nat.Sampler(N, D, flags=nat.FLAG_DEFER_REDISTRIBUTE, **kw)


def _bits(t):
    t = t.detach().contiguous()
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu()


def _state(S):
    x, lp = S.current()  # (completes a pending redistribution)
    return _bits(x), _bits(lp), _bits(S.logw)


def _assert_same_state(a, b):
    for u, v in zip(_state(a), _state(b)):
        assert torch.equal(u, v)


def _assert_same_outputs(ra, rb):
    for key in ("mean", "fhat", "trace"):
        if ra[key] is not None:
            assert torch.equal(_bits(ra[key]), _bits(rb[key])), key


@pytest.mark.parametrize("N,D,mode", [(70001, 16, 1), (4097, 5, 1), (100003, 8, 0), (1 << 20, 16, 0),
                                      (9000, 12, 1), (8193, 1, 1)])
def test_defer_one_call_bit_identical(nat, N, D, mode):
    A, B = _pair(nat, N, D, mode)
    ra = A.step(6, trace=True, fhat=True)
    rb = B.step(6, trace=True, fhat=True)
    A.sync()
    B.sync()
    _assert_same_outputs(ra, rb)
    _assert_same_state(A, B)
    tr = nat.trace_dicts(rb["trace"])
    if mode == 1:
        assert all(t["resampled"] == 1 for t in tr)


@pytest.mark.parametrize("mode", [0, 1])
def test_defer_across_calls(nat, mode):
    """The redistribution stays pending between calls: single iterations,
    profiled iterations and multi-iteration calls in a row."""
    N, D = 50003, 16
    A, B = _pair(nat, N, D, mode, seed=7)
    ra = A.step(8, trace=True, fhat=True)
    for _ in range(3):
        B.step(1)
    B.step_profile()
    B.step_profile()
    rb = B.step(3, trace=True, fhat=True)
    A.sync()
    B.sync()
    assert torch.equal(_bits(ra["mean"]), _bits(rb["mean"]))
    assert torch.equal(_bits(ra["fhat"]), _bits(rb["fhat"]))
    assert torch.equal(_bits(ra["trace"][-3:]), _bits(rb["trace"]))
    _assert_same_state(A, B)


def test_defer_heavy_duplication(nat):
    """A narrow target far from the initial cloud: few survivors, runs of
    thousands of copies spanning several copy tiles, so most move tiles take
    their first source from the copy-tile starts after a long backward
    search."""
    N, D = 60001, 4
    mu = np.full(D, 3.0)
    sigma = np.eye(D) * 0.05
    A, B = _pair(nat, N, D, 1, seed=11, mu=mu, sigma=sigma)
    ra = A.step(4, trace=True)
    rb = B.step(4, trace=True)
    A.sync()
    B.sync()
    surv = [t["survivors"] for t in nat.trace_dicts(rb["trace"])]
    assert min(surv) < N // 20, surv
    _assert_same_outputs(ra, rb)
    _assert_same_state(A, B)


def test_defer_then_other_calls(nat):
    """Any other call completes the pending redistribution first: the
    piecewise stages after deferred steps, and a checkpoint taken while one is
    pending, restored into a new deferred sampler that continues."""
    N, D = 30011, 16
    A, B = _pair(nat, N, D, 1, seed=5)
    A.step(3)
    B.step(3)
    for S in (A, B):
        S.move()
        S.reweight()
        nc, _ = S.resample()
        S.redistribute(nc)
    A.sync()
    B.sync()
    _assert_same_state(A, B)
    ma, _ = A.estimate()
    mb, _ = B.estimate()
    assert torch.equal(_bits(ma), _bits(mb))
    B.step(2)
    blob = B.checkpoint()
    mu, sigma = inputs.gaussian_target(D, seed=D)
    C = nat.Sampler(N, D, dtype=torch.float32, seed=5, mu=mu, sigma=sigma, step=0.5, resample_mode=1,
                    flags=nat.FLAG_DEFER_REDISTRIBUTE)
    C.restore(blob)
    ra = A.step(4, trace=True)
    rc = C.step(2, trace=True)
    B.step(2)
    A.sync()
    C.sync()
    assert torch.equal(_bits(ra["mean"]), _bits(rc["mean"]))
    assert torch.equal(_bits(ra["trace"][-2:]), _bits(rc["trace"]))
    _assert_same_state(A, C)
    _assert_same_state(A, B)


def test_defer_full_size(nat):
    """The headline shape, N = 2^22, D = 16, resampling every iteration."""
    N, D = 1 << 22, 16
    A, B = _pair(nat, N, D, 1, seed=2)
    ra = A.step(3, trace=True, fhat=True)
    rb = B.step(3, trace=True, fhat=True)
    A.sync()
    B.sync()
    _assert_same_outputs(ra, rb)
    _assert_same_state(A, B)


@pytest.mark.parametrize("N,D,dtype", [(4096, 16, torch.float32), (20000, 32, torch.float32),
                                       (20000, 4, torch.float64)])
def test_defer_flag_ignored_where_not_honoured(nat, N, D, dtype):
    """One quantise block, D > 16, FP64: the flag is ignored, results equal."""
    mu, sigma = inputs.gaussian_target(D, seed=D)
    kw = dict(dtype=dtype, seed=9, mu=mu, sigma=sigma, resample_mode=1)
    A = nat.Sampler(N, D, **kw)
    B = nat.Sampler(N, D, flags=nat.FLAG_DEFER_REDISTRIBUTE, **kw)
    ra = A.step(3, trace=True)
    rb = B.step(3, trace=True)
    A.sync()
    B.sync()
    _assert_same_outputs(ra, rb)
    _assert_same_state(A, B)
