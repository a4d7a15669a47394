"""FP64 samplers of at most 2048 particles run smc_step's iterations in one
cooperative launch: every block moves and reweights its particles (the
separate move launch's particle-to-thread map), then block 0 runs the
maximum, the quantise / scan pass, the copy and the commit (Algorithm 2,
lines 3-10), with grid barriers between the phases.  The stage bodies are
those of the separate launches, so the results must equal, bit for bit,
the same iterations launched stage by stage (smc_step_profile) and the
oracle's run; a barrier that never completes must time out, be reported as
SMC_ETIMEOUT, and leave the context usable."""
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


def host(t):
    return t.detach().cpu().numpy()


def _bits(t):
    t = t.detach().contiguous()
    return t.view(torch.int64 if t.element_size() == 8 else torch.int32).cpu()


def _make(nat, n, d, seed, mode, **kw):
    mu, sig = inputs.gaussian_target(d, seed=40 + d)
    return nat.Sampler(n, d, dtype=torch.float64, seed=seed, mu=mu, sigma=sig, step=0.5, init_scale=2.0,
                       resample_mode=mode, **kw)


def _state(S):
    x, lp = S.current()
    return _bits(x), _bits(lp), _bits(S.logw)


# (N, D): one particle, ragged sizes, the largest size the fused path takes
# (one copy tile), and every width class of its kernel
CASES = [(1024, 4), (2048, 8), (1, 1), (5, 3), (777, 2), (1500, 16), (2000, 32), (64, 5), (2047, 12)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,d", CASES)
def test_fused_equals_stage_launches(nat, n, d, mode):
    K = 9
    a = _make(nat, n, d, 11, mode)
    b = _make(nat, n, d, 11, mode)
    ra = a.step(K, trace=True)
    for _ in range(K):
        b.step_profile()
    a.sync()
    b.sync()
    for u, v in zip(_state(a), _state(b)):
        assert torch.equal(u, v), (n, d, mode)
    sa, sb = a.stats(), b.stats()
    for key in ("lse", "logc", "ess", "max_logw", "resampled", "t", "survivors"):
        assert sa[key] == sb[key] or (np.isnan(sa[key]) and np.isnan(sb[key])), key
    tr = nat.trace_dicts(ra["trace"])
    assert [r["t"] for r in tr] == list(range(1, K + 1))
    assert tr[-1]["lse"] == sa["lse"] and tr[-1]["resampled"] == sa["resampled"]
    if mode == 1:
        assert all(r["resampled"] == 1 for r in tr)
    a.close()
    b.close()


def test_fused_calls_continue_the_chain(nat):
    # the barrier is reset per call and t is read from the device: 5 + 4
    # iterations in two calls equal 9 in one
    a = _make(nat, 1024, 4, 3, 0)
    b = _make(nat, 1024, 4, 3, 0)
    a.step(5)
    r2 = a.step(4, trace=True)
    b.step(9)
    a.sync()
    b.sync()
    for u, v in zip(_state(a), _state(b)):
        assert torch.equal(u, v)
    assert [r["t"] for r in nat.trace_dicts(r2["trace"])] == [6, 7, 8, 9]


@pytest.mark.parametrize("n,d,seed", [(2048, 8, 3), (333, 1, 5), (1000, 6, 7)])
def test_fused_against_oracle(nat, orc, n, d, seed):
    # as the C0 end-to-end test, at other sizes: particles, log pi and log w
    # bit for bit, the statistics within the FP64 tolerances
    K = 12
    mu, sig = inputs.gaussian_target(d, seed=40 + d)
    ref = orc.run(orc.Target.gauss(mu, sig), n, seed, K, init_scale=2.0, step=0.5, ncopies_trace=True)
    S = _make(nat, n, d, seed, 0)
    out = S.step(K, cov=True, trace=True, fhat=True)
    S.sync()
    x, lp = S.current()
    assert np.array_equal(host(x), ref["x"])
    assert np.array_equal(host(lp), ref["logpi"])
    assert np.array_equal(host(S.logw), ref["logw"])
    tr = nat.trace_dicts(out["trace"])
    for k in range(K):
        assert tr[k]["resampled"] == int(ref["trace"][k, 4]), k
        assert abs(tr[k]["lse"] - ref["trace"][k, 0]) <= 1e-10, k
        assert tr[k]["max_logw"] == ref["trace"][k, 3], k
        assert tr[k]["survivors"] == int(ref["trace"][k, 5]), k
    np.testing.assert_allclose(host(out["mean"]), ref["means"][-1], rtol=0, atol=1e-11)
    np.testing.assert_allclose(host(out["cov"]), ref["cov"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(host(out["fhat"]), ref["fhat"], rtol=0, atol=1e-10)
    S.close()


def test_stalled_barrier_times_out_and_the_context_survives(nat):
    """Failure path without a GPU fault: with the test hook the grid barrier
    waits for one block more than the launch has, every wait runs out after
    about half a second, the kernel returns, and smc_sync reports
    SMC_ETIMEOUT.  A normal sampler then runs on the same context."""
    S = _make(nat, 256, 2, 1, 0, flags=nat.FLAG_TEST_STALL_BARRIER)
    S.step(3)
    with pytest.raises(nat.SmcError) as e:
        S.sync()
    assert e.value.code == nat.SMC_ETIMEOUT
    S.sync()  # cleared
    S.close()
    T = _make(nat, 256, 2, 1, 0)
    r = T.step(3)
    T.sync()
    assert np.all(np.isfinite(host(r["mean"])))
    T.close()
