"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Bit-exact: copy counts, redistributed rows, the quantised sums and decision,
and -- on the FP64 path, whose element-wise arithmetic is a fixed sequence of
IEEE operations on both sides -- particles, log-weights and log-targets over a
whole run.  Tolerances (floating-point reductions, FP32 state):
  LSE, log c_t          |d| <= 1e-10   (exact integer sums on the GPU; the gap is
                                        the oracle's own FP64 summation error plus
                                        the terms below 2^-62 that quantise to 0)
  N_eff                 rel <= 1e-9    (FP64 path; quantised vs plain weights)
  mean, recycled mean   |d| <= 1e-11   (FP64 path)
  covariance            |d| <= 1e-9    (FP64 path)
  FP32 state            |d| <= 4e-6 (1 + |x|) for moved particles, rel 2e-5 for
                        log pi, 2e-4 relative for weights (the reduced-precision
                        bound of the specification)
"""
import math

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


DEV = "cuda"


def to_dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ redistribute
ROW_TYPES = [(np.float32, 16), (np.float32, 1), (np.float32, 2), (np.float32, 3), (np.float64, 4),
             (np.float32, 32), (np.float64, 32), (np.float32, 5)]


@pytest.mark.parametrize("N", [1, 2, 7, 4095, 4096, 4097, 12289, 100003])
@pytest.mark.parametrize("kind", ["multinomial", "skewed", "one_hot", "ones"])
def test_redistribute_raw_bit_exact(nat, orc, N, kind):
    nc = inputs.composition(N, seed=N, kind=kind)
    ncd = to_dev(nc)
    for dt, D in ROW_TYPES:
        x = inputs.particles(N, D, seed=D, dtype=dt)
        out = nat.smc_redistribute_raw(ncd, to_dev(x))
        torch.cuda.synchronize()
        ref = orc.redistribute(nc, x)
        assert np.array_equal(host(out).view(np.uint8), ref.view(np.uint8)), (dt, D)


def test_redistribute_raw_rejects_bad_ncopies(nat):
    N = 5000
    x = to_dev(inputs.particles(N, 16, seed=1))
    for bad in ("sum", "negative"):
        nc = inputs.composition(N, seed=2)
        if bad == "sum":
            nc[0] += 1
        else:
            j, k = int(np.argmax(nc)), int(np.argmin(nc))
            nc[j] += 1
            nc[k] -= 1
            assert nc.sum() == N and nc.min() < 0
        ws = torch.empty(nat.smc_redistribute_ws_bytes(N), dtype=torch.uint8, device=DEV)
        out = torch.full_like(x, 7.0)
        nat.smc_redistribute_raw(to_dev(nc), x, out, ws=ws)
        assert nat.smc_ws_status(ws) == nat.SMC_EINVAL
        assert torch.all(out == 7.0)
        # the workspace is usable again afterwards
        good = to_dev(inputs.composition(N, seed=3))
        nat.smc_redistribute_raw(good, x, out, ws=ws)
        assert nat.smc_ws_status(ws) == nat.SMC_OK


def test_redistribute_raw_repeatable(nat):
    N = 300001
    nc = to_dev(inputs.composition(N, seed=9, kind="skewed"))
    x = to_dev(inputs.particles(N, 16, seed=9))
    a = nat.smc_redistribute_raw(nc, x)
    b = nat.smc_redistribute_raw(nc, x)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# ------------------------------------------------------------------ resample
def _logw_cases(N):
    yield "s0.5", inputs.log_weights(N, 0.5, seed=N)
    yield "s2", inputs.log_weights(N, 2.0, seed=N + 1)
    yield "s8", inputs.log_weights(N, 8.0, seed=N + 2)
    yield "onehot", inputs.one_hot_log_weights(N, seed=N)
    yield "equal", np.full(N, -1.25)
    lw = inputs.log_weights(N, 3.0, seed=N + 3)
    lw[::3] = -np.inf
    if N > 1:
        yield "someinf", lw
    yield "shifted", inputs.log_weights(N, 1.0, seed=N + 4) - 1e4


@pytest.mark.parametrize("N", [1, 2, 3, 1000, 4097, 65553])
@pytest.mark.parametrize("mode", [0, 1])
def test_resample_raw_bit_exact(nat, orc, N, mode):
    for name, lw in _logw_cases(N):
        seed, t = 17, 5
        nc, st = nat.smc_resample_raw(to_dev(lw), seed, t, mode)
        torch.cuda.synchronize()
        s = nat.decode_stats(st)
        r = orc.resample(lw, seed, t, mode)
        nc_ref, _ = orc.systematic(r["W"], r["S"], r["U"])
        assert np.array_equal(host(nc), nc_ref), name
        assert host(nc).sum() == N
        assert s["resampled"] == int(r["did"]), name
        assert s["max_logw"] == r["m"]
        m, lse, ess = orc.lse_ess(lw)
        assert abs(s["lse"] - lse) <= 1e-10 + 1e-15 * abs(lse), (name, s["lse"], lse)
        ess_q = r["S"] ** 2 / r["sumW2"]
        assert abs(s["ess"] - ess_q) <= 1e-12 * ess_q, name
        assert abs(s["ess"] - ess) <= 1e-6 * ess, name


def test_resample_raw_nonfinite(nat):
    N = 777
    ws = torch.empty(nat.smc_redistribute_ws_bytes(N), dtype=torch.uint8, device=DEV)
    lw = np.zeros(N)
    lw[100] = np.nan
    nat.smc_resample_raw(to_dev(lw), 1, 1, 1, ws=ws)
    assert nat.smc_ws_status(ws) == nat.SMC_ENONFINITE
    nat.smc_resample_raw(to_dev(np.full(N, -np.inf)), 1, 1, 1, ws=ws)
    assert nat.smc_ws_status(ws) == nat.SMC_ENONFINITE
    nat.smc_resample_raw(to_dev(np.zeros(N)), 1, 1, 1, ws=ws)
    assert nat.smc_ws_status(ws) == nat.SMC_OK


# ------------------------------------------------------------------ sampler, FP64
def _gauss(D, seed=0):
    mu, Sigma = inputs.gaussian_target(D, seed=seed)
    return mu, Sigma


@pytest.mark.parametrize("N,D", [(1000, 4), (4099, 3), (1, 2), (257, 16)])
def test_fp64_stages_bit_exact(nat, orc, N, D):
    mu, Sigma = _gauss(D, seed=D)
    tgt = orc.Target.gauss(mu, Sigma)
    seed, step, s0 = 11, 0.5, 2.0
    S = nat.Sampler(N, D, dtype=torch.float64, seed=seed, mu=mu, sigma=Sigma, step=step, init_scale=s0,
                    resample_mode=nat.RESAMPLE_ALWAYS)
    x0, lw0, lp0 = orc.init(tgt, N, seed, s0)
    xg, lpg = S.current()
    assert np.array_equal(host(xg), x0)
    assert np.array_equal(host(S.logw), lw0)
    assert np.array_equal(host(lpg), lp0)
    # Algorithm 2 line 4: move, then eq. (5)
    S.move()
    x1 = orc.move(x0, seed, 1, step)
    xg, lpg = S.current()
    assert np.array_equal(host(xg), x1)
    S.reweight()
    lw1, lp1 = orc.reweight(tgt, x0, x1, lp0, lw0, step)
    assert np.array_equal(host(S.logw), lw1)
    assert np.array_equal(host(lpg), lp1)
    st = S.stats()
    m, lse, ess = orc.lse_ess(lw1)
    assert st["max_logw"] == m
    assert abs(st["lse"] - lse) <= 1e-10
    assert abs(st["ess"] - ess) <= 1e-9 * ess
    # eq. (7)
    mean, cov = S.estimate(cov=True)
    mref, cref = orc.estimate(x1, lw1, lse)
    np.testing.assert_allclose(host(mean), mref, rtol=0, atol=1e-11)
    np.testing.assert_allclose(host(cov), cref, rtol=0, atol=1e-9)
    # Algorithm 4: MVR, S-R, reset
    nc, did = S.resample()
    r = orc.resample(lw1, seed, 1, orc.RESAMPLE_ALWAYS)
    assert int(host(did)[0]) == 1
    assert np.array_equal(host(nc), r["ncopies"])
    S.redistribute(nc)
    xg, lpg = S.current()
    assert np.array_equal(host(xg), orc.redistribute(r["ncopies"], x1))
    assert np.array_equal(host(lpg), orc.redistribute(r["ncopies"], lp1))
    assert np.all(host(S.logw) == orc.reset_logw(N))
    S.sync()
    S.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_fp64_end_to_end_C0(nat, orc, seed):
    # the plain FP64 sampler: N=1024, D=4, K=20, step 0.5, q0 = N(0, 4I), ESS < N/2
    N, D, K = 1024, 4, 20
    mu, Sigma = _gauss(D, seed=0)
    tgt = orc.Target.gauss(mu, Sigma)
    ref = orc.run(tgt, N, seed, K, init_scale=2.0, step=0.5, ncopies_trace=True)
    S = nat.Sampler(N, D, dtype=torch.float64, seed=seed, mu=mu, sigma=Sigma, step=0.5, init_scale=2.0)
    out = S.step(K, cov=True, trace=True, fhat=True)
    S.sync()
    x, lp = S.current()
    assert np.array_equal(host(x), ref["x"])
    assert np.array_equal(host(S.logw), ref["logw"])
    assert np.array_equal(host(lp), ref["logpi"])
    tr = nat.trace_dicts(out["trace"])
    for k in range(K):
        assert tr[k]["t"] == k + 1
        assert tr[k]["resampled"] == int(ref["trace"][k, 4]), k
        assert abs(tr[k]["lse"] - ref["trace"][k, 0]) <= 1e-10, k
        assert abs(tr[k]["logc"] - ref["trace"][k, 1]) <= 1e-10, k
        assert abs(tr[k]["ess"] - ref["trace"][k, 2]) <= 1e-9 * ref["trace"][k, 2], k
        assert tr[k]["max_logw"] == ref["trace"][k, 3], k
        assert tr[k]["survivors"] == int(ref["trace"][k, 5]), k
    np.testing.assert_allclose(host(out["mean"]), ref["means"][-1], rtol=0, atol=1e-11)
    np.testing.assert_allclose(host(out["cov"]), ref["cov"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(host(out["fhat"]), ref["fhat"], rtol=0, atol=1e-10)
    S.close()


def test_graph_and_direct_launches_agree(nat):
    N, D, K = 3001, 4, 7
    mu, Sigma = _gauss(D)
    a = nat.Sampler(N, D, dtype=torch.float64, seed=5, mu=mu, sigma=Sigma)
    b = nat.Sampler(N, D, dtype=torch.float64, seed=5, mu=mu, sigma=Sigma, stream=torch.cuda.default_stream())
    ra = a.step(K, trace=True)
    rb = b.step(K, trace=True)
    a.sync()
    b.sync()
    assert torch.equal(a.current()[0], b.current()[0])
    assert torch.equal(ra["trace"], rb["trace"])
    # repeated calls continue the same chain (graph replay reads t from the device)
    ra2 = a.step(3, trace=True)
    rb2 = b.step(3, trace=True)
    assert torch.equal(ra2["trace"], rb2["trace"])
    assert nat.trace_dicts(ra2["trace"])[0]["t"] == K + 1


def test_nonfinite_weights_reported(nat):
    N, D = 100, 2
    S = nat.Sampler(N, D, dtype=torch.float64, seed=1, mu=np.zeros(D), sigma=np.eye(D))
    S.logw.fill_(float("nan"))
    S.reweight()
    with pytest.raises(nat.SmcError) as e:
        S.sync()
    assert e.value.code == nat.SMC_ENONFINITE
    S.sync()  # cleared


# ------------------------------------------------------------------ sampler, FP32
@pytest.mark.parametrize("N,D", [(5003, 16), (4096, 2), (999, 8), (2049, 32), (3001, 12), (777, 10), (1500, 20),
                                 (257, 5)])
def test_fp32_stages(nat, orc, N, D):
    mu, Sigma = _gauss(D, seed=D)
    tgt = orc.Target.gauss(mu, Sigma)
    seed, step = 21, 0.5
    S = nat.Sampler(N, D, dtype=torch.float32, seed=seed, mu=mu, sigma=Sigma, step=step,
                    resample_mode=nat.RESAMPLE_ALWAYS)
    x0g, lp0g = [host(t).copy() for t in S.current()]
    lw0g = host(S.logw).copy()
    x0, lw0, lp0 = orc.init(tgt, N, seed, 2.0, ubits=24)
    assert np.all(np.abs(x0g - x0) <= 4e-6 * (1 + np.abs(x0)))
    lp_of_g = tgt.logpi(x0g.astype(np.float64))
    assert np.all(np.abs(lp0g - lp_of_g) <= 2e-5 * (1 + np.abs(lp_of_g)))
    q0 = -0.5 * np.sum(x0g.astype(np.float64) ** 2, axis=1) / 4.0
    assert np.all(np.abs(lw0g - (lp_of_g - q0)) <= 2e-4 * (1 + np.abs(lp_of_g - q0)))
    S.move()
    x1g = host(S.current()[0]).copy()
    x1 = orc.move(x0g.astype(np.float64), seed, 1, step, ubits=24)
    assert np.all(np.abs(x1g - x1) <= 4e-6 * (1 + np.abs(x1)))
    S.reweight()
    x1g, lp1g = [host(t).copy() for t in S.current()]
    lw1g = host(S.logw).copy()
    lp_ref = tgt.logpi(x1g.astype(np.float64))
    assert np.all(np.abs(lp1g - lp_ref) <= 2e-5 * (1 + np.abs(lp_ref)))
    # eq. (5) with the GPU's own FP32 log pi values: the difference in FP32,
    # the accumulation in FP64
    np.testing.assert_array_equal(lw1g, lw0g + (lp1g.astype(np.float32) - lp0g.astype(np.float32)).astype(np.float64))
    st = S.stats()
    m, lse, ess = orc.lse_ess(lw1g)
    assert st["max_logw"] == m
    assert abs(st["lse"] - lse) <= 1e-10
    mean, _ = S.estimate()
    mref, _ = orc.estimate(x1g.astype(np.float64), lw1g, lse, with_cov=False)
    np.testing.assert_allclose(host(mean), mref, rtol=0, atol=2e-5 * (1 + np.abs(mref).max()))
    nc, did = S.resample()
    r = orc.resample(lw1g, seed, 1, orc.RESAMPLE_ALWAYS)
    assert np.array_equal(host(nc), r["ncopies"])
    S.redistribute(nc)
    x2g, lp2g = [host(t) for t in S.current()]
    assert np.array_equal(x2g, orc.redistribute(r["ncopies"], x1g))
    assert np.array_equal(lp2g, orc.redistribute(r["ncopies"], lp1g))
    S.sync()


@pytest.mark.parametrize("step", [0.05, 0.3, 1.7])
@pytest.mark.parametrize("N,D", [(4099, 16), (1025, 5)])
def test_fp32_move_step_sizes(nat, orc, N, D, step):
    """The FP32 move folds the step into its Box-Muller constants (eps^2 in
    the radius, -eps r in the two FMAs); steps whose square is not a power of
    two round there, on the vector (D = 16) and scalar (D = 5) row paths.
    The bound scales with the step: the normals' own error is a few 1e-6."""
    mu, Sigma = _gauss(D, seed=D)
    seed = 33
    S = nat.Sampler(N, D, dtype=torch.float32, seed=seed, mu=mu, sigma=Sigma, step=step,
                    resample_mode=nat.RESAMPLE_ALWAYS)
    x0g = host(S.current()[0]).copy()
    S.move()
    x1g = host(S.current()[0]).copy()
    x1 = orc.move(x0g.astype(np.float64), seed, 1, step, ubits=24)
    tol = 4e-6 * max(1.0, 2.0 * step) * (1 + np.abs(x1))
    assert np.all(np.abs(x1g - x1) <= tol)
    S.sync()


def test_fp32_step_equals_piecewise(nat):
    N, D = 70001, 16
    mu, Sigma = _gauss(D)
    kw = dict(dtype=torch.float32, seed=3, mu=mu, sigma=Sigma, resample_mode=nat.RESAMPLE_ALWAYS)
    a = nat.Sampler(N, D, **kw)
    b = nat.Sampler(N, D, **kw)
    for _ in range(3):
        a.step(1)
        b.move()
        b.reweight()
        nc, _ = b.resample()
        b.redistribute(nc)
    a.sync()
    b.sync()
    assert torch.equal(a.current()[0], b.current()[0])
    assert torch.equal(a.current()[1], b.current()[1])
    assert torch.equal(a.logw, b.logw)


def test_fp32_posterior_moments(nat):
    # batched-sampler shape: FP32 state, D=8, moments against the closed form
    D, N, K = 8, 1 << 16, 30
    mu, Sigma = _gauss(D, seed=8)
    est = []
    for seed in range(8):
        S = nat.Sampler(N, D, dtype=torch.float32, seed=seed, mu=mu, sigma=Sigma)
        out = S.step(K, fhat=True)
        est.append(host(out["fhat"]))
    est = np.array(est)
    se = est.std(axis=0, ddof=1) / math.sqrt(len(est))
    z = (est.mean(axis=0) - mu) / np.maximum(se, 1e-3)
    assert np.all(np.abs(z) < 5.0), z


# ------------------------------------------------------------------ full size
def test_full_size_resample_redistribute(nat, orc):
    # the microbenchmark's largest size: N = 2^24, D = 16 FP32 rows
    N, D = 1 << 24, 16
    lw = inputs.log_weights(N, 2.0, seed=0)
    nc, st = nat.smc_resample_raw(to_dev(lw), 0, 1, nat.RESAMPLE_ALWAYS)
    torch.cuda.synchronize()
    r = orc.resample(lw, 0, 1, orc.RESAMPLE_ALWAYS)
    ncg = host(nc)
    assert np.array_equal(ncg, r["ncopies"])
    x = inputs.particles(N, D, seed=1)
    out = host(nat.smc_redistribute_raw(nc, to_dev(x)))
    # sampled outputs: row k is row src(k), src(k) = #{i : csum_i <= k}
    csum = np.cumsum(ncg.astype(np.int64))
    ks = np.random.default_rng(0).integers(0, N, 200000)
    ks = np.concatenate([ks, [0, N - 1, 4095, 4096, 4097]])
    src = np.searchsorted(csum, ks, side="right")
    assert np.array_equal(out[ks], x[src])


def test_full_size_iteration_sampled(nat, orc):
    # one iteration at N = 2^24, D = 16 (FP32), resampling every iteration,
    # checked on sampled particles that the oracle recomputes one by one
    N, D = 1 << 24, 16
    mu, Sigma = _gauss(D, seed=16)
    tgt = orc.Target.gauss(mu, Sigma)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=4, mu=mu, sigma=Sigma, resample_mode=nat.RESAMPLE_ALWAYS)
    ids = np.random.default_rng(1).integers(0, N, 3000)
    x0 = host(S.current()[0])[ids].astype(np.float64)
    lw0 = host(S.logw)[ids]
    lp0 = host(S.current()[1])[ids]
    S.move()
    S.reweight()
    x1g, lp1g = [host(t) for t in S.current()]
    lw1g = host(S.logw)
    # move of particle i depends only on (seed, t, i, x_i)
    for j, i in enumerate(ids[:300]):
        z = orc.normals(4, 1, orc.ORC_MOVE, int(i), D, 24)
        assert np.all(np.abs(x1g[i] - (x0[j] + 0.5 * z)) <= 4e-6 * (1 + np.abs(x0[j])))
    lp_ref = tgt.logpi(x1g[ids].astype(np.float64))
    assert np.all(np.abs(lp1g[ids] - lp_ref) <= 2e-5 * (1 + np.abs(lp_ref)))
    np.testing.assert_array_equal(lw1g[ids], lw0 + (lp1g[ids].astype(np.float32) - lp0.astype(np.float32)).astype(np.float64))
    nc, _ = S.resample()
    r = orc.resample(lw1g, 4, 1, orc.RESAMPLE_ALWAYS)
    ncg = host(nc)
    assert np.array_equal(ncg, r["ncopies"])
    S.redistribute(nc)
    x2g = host(S.current()[0])
    csum = np.cumsum(ncg.astype(np.int64))
    ks = np.random.default_rng(2).integers(0, N, 100000)
    assert np.array_equal(x2g[ks], x1g[np.searchsorted(csum, ks, side="right")])
    assert np.all(host(S.logw[:: 4097]) == orc.reset_logw(N))
    S.sync()


@pytest.mark.parametrize("D", [3, 8, 16])
def test_fp32_mean_from_move_records_matches_rows(nat, D):
    """After a resampling iteration every log w is the same, and the fused
    move kernel forms the eq. (7) sums itself (per 256-particle tile, from
    the FP32 log pi differences); the piecewise path forms them from the
    rows in the quantise pass.  Same particles and weights, two summation
    routes: the means agree to FP32 rounding."""
    N = 300007
    mu, Sigma = _gauss(D)
    kw = dict(dtype=torch.float32, seed=9, mu=mu, sigma=Sigma, resample_mode=nat.RESAMPLE_ALWAYS, step=0.3)
    a = nat.Sampler(N, D, **kw)
    b = nat.Sampler(N, D, **kw)
    for it in range(4):
        ra = a.step(1)
        b.move()
        b.reweight()
        mb, _ = b.estimate()
        nc, _ = b.resample()
        b.redistribute(nc)
        a.sync()
        b.sync()
        assert torch.equal(a.logw, b.logw)
        scale = 1.0 + mb.abs()
        assert torch.all((ra["mean"] - mb).abs() <= 1e-5 * scale), (it, ra["mean"], mb)


@pytest.mark.parametrize("frac", [0.25, 0.75, 1.0])
def test_fp64_run_with_threshold_nstar(nat, orc, frac):
    """Algorithm 2 with its threshold input N* (resample iff N_eff < N*):
    a whole FP64 run against the oracle's with the same N*, decisions and
    particles bit for bit; N* = N/4 resamples less and 3N/4 more often than
    the default N/2."""
    N, D, K = 1024, 4, 12
    nstar = int(frac * N)
    mu, Sigma = _gauss(D, seed=0)
    tgt = orc.Target.gauss(mu, Sigma)
    ref = orc.run(tgt, N, 3, K, init_scale=2.0, step=0.5, nstar=nstar)
    S = nat.Sampler(N, D, dtype=torch.float64, seed=3, mu=mu, sigma=Sigma, step=0.5, init_scale=2.0, nstar=nstar)
    out = S.step(K, trace=True)
    S.sync()
    tr = nat.trace_dicts(out["trace"])
    assert [t["resampled"] for t in tr] == [int(v) for v in ref["trace"][:, 4]]
    x, lp = S.current()
    assert np.array_equal(host(x), ref["x"])
    assert np.array_equal(host(S.logw), ref["logw"])
    # the decision is N_eff < N* on the quantised weights
    for t in tr:
        assert t["resampled"] == int(t["ess"] < nstar) or abs(t["ess"] - nstar) < 1e-9 * nstar
    S.close()


def test_fp32_threshold_rejects_out_of_range(nat):
    mu, Sigma = _gauss(2)
    with pytest.raises(nat.SmcError) as e:
        nat.Sampler(100, 2, dtype=torch.float32, mu=mu, sigma=Sigma, nstar=101)
    assert e.value.code == nat.SMC_EINVAL


def test_redistribute_raw_profile_same_output(nat, orc):
    """The profiled stateless call writes the same rows as the plain one and
    records its three events in order (scan before copy)."""
    N = 100003
    nc = inputs.composition(N, seed=21)
    x = np.random.default_rng(22).standard_normal((N, 16)).astype(np.float32)
    ncd, xd = torch.as_tensor(nc, device="cuda"), torch.as_tensor(x, device="cuda")
    ws = torch.empty(nat.smc_redistribute_ws_bytes(N), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(xd)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    nat.smc_redistribute_raw_profile(ncd, xd, out, ws, evs)
    torch.cuda.synchronize()
    assert nat.smc_ws_status(ws) == nat.SMC_OK
    assert np.array_equal(out.cpu().numpy(), orc.redistribute(nc, x))
    assert evs[0].elapsed_time(evs[1]) >= 0 and evs[1].elapsed_time(evs[2]) > 0


@pytest.mark.parametrize("D", [2, 16, 32])
def test_fp32_covariance_against_oracle(nat, orc, D):
    """The weighted covariance of eq. (7)'s estimate (the diagnostic output)
    for FP32 state against the oracle's on the same particles and weights."""
    N = 40000
    mu, Sigma = _gauss(D, seed=3)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=5, mu=mu, sigma=Sigma, resample_mode=nat.RESAMPLE_NEVER)
    S.move()
    S.reweight()
    mean, cov = S.estimate(cov=True)
    S.sync()
    x = host(S.current()[0]).astype(np.float64)
    lw = host(S.logw)
    _, lse, _ = orc.lse_ess(lw)
    mref, cref = orc.estimate(x, lw, lse, with_cov=True)
    scale = 1.0 + np.abs(cref).max()
    np.testing.assert_allclose(host(cov), cref, rtol=0, atol=5e-5 * scale)
    np.testing.assert_allclose(host(mean), mref, rtol=0, atol=2e-5 * (1 + np.abs(mref).max()))
    c = host(cov)
    assert np.array_equal(c, c.T)


@pytest.mark.parametrize("N", [4097, 100003])
def test_redistribute_raw_misaligned_ncopies(nat, orc, N):
    """A copy-count vector that does not start on a 16-byte boundary (a
    slice of a larger tensor) takes the scalar-load path: same rows."""
    nc = inputs.composition(N, seed=N + 5)
    x = np.random.default_rng(N).standard_normal((N, 16)).astype(np.float32)
    big = torch.zeros(N + 3, dtype=torch.int32, device="cuda")
    big[1:N + 1] = torch.as_tensor(nc, device="cuda")
    ncd = big[1:N + 1]
    assert ncd.data_ptr() % 16 != 0
    ws = torch.empty(nat.smc_redistribute_ws_bytes(N), dtype=torch.uint8, device="cuda")
    out = nat.smc_redistribute_raw(ncd, torch.as_tensor(x, device="cuda"), ws=ws)
    torch.cuda.synchronize()
    assert nat.smc_ws_status(ws) == nat.SMC_OK
    assert np.array_equal(out.cpu().numpy(), orc.redistribute(nc, x))
