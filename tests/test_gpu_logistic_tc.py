"""The tensor-core logistic likelihood (tcgen05 BF16 hi / lo split, FP32
accumulation in TMEM, MUFU epilogue) against the FP64 oracle.

Error budget per particle: the split drops only B_lo X_lo (2^-16 of each
product) and FP32 accumulation adds ~2^-24 per term, so |dz| is about
|z| 2^-16 at worst; the epilogue's ex2 / lg2 approximations add ~1e-7 per
row.  Over M rows the log-target error stays far below the reduced-precision
bound used for every FP32 stage: |d log pi| <= 2e-5 (1 + |log pi|).  The test
also records the worst absolute error it saw (printed with -s).
"""
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


CASES = [(1000, 5, 300), (129, 32, 257), (1, 3, 1), (4096, 32, 8192), (777, 16, 1000), (20000, 8, 2048)]


@pytest.mark.parametrize("N,D,M", CASES)
def test_tc_logpi_against_oracle(nat, orc, N, D, M):
    X, y, _ = inputs.logistic_data(M, D, seed=M + D)
    tgt = orc.Target.logistic(X.astype(np.float64), y.astype(np.float64), 4.0)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=7, target="logistic", X=X, y=y, prior_var=4.0, step=0.2,
                    resample_mode=nat.RESAMPLE_NEVER)
    x0, lp0 = [host(t).copy() for t in S.current()]
    ref0 = tgt.logpi(x0.astype(np.float64))
    err0 = np.abs(lp0 - ref0)
    assert np.all(err0 <= 2e-5 * (1 + np.abs(ref0))), err0.max()
    lw0 = host(S.logw).copy()
    S.move()
    S.reweight()
    x1, lp1 = [host(t).copy() for t in S.current()]
    lw1 = host(S.logw)
    ref1 = tgt.logpi(x1.astype(np.float64))
    err1 = np.abs(lp1 - ref1)
    assert np.all(err1 <= 2e-5 * (1 + np.abs(ref1))), err1.max()
    # eq. (5) with the stored FP32 log pi values
    np.testing.assert_array_equal(lw1, lw0 + (lp1 - lp0).astype(np.float64))
    S.sync()
    print(f"N={N} D={D} M={M}: max |d log pi| = {max(err0.max(), err1.max()):.3e} "
          f"(|log pi| up to {np.abs(ref1).max():.1f})")


def test_tc_matches_cuda_cores(nat, orc):
    """Same particles (the initial draw does not depend on the likelihood
    path): tensor-core and CUDA-core FP32 log pi agree within the bound."""
    N, D, M = 3000, 32, 4096
    X, y, _ = inputs.logistic_data(M, D, seed=5)
    a = nat.Sampler(N, D, dtype=torch.float32, seed=2, target="logistic", X=X, y=y)
    b = nat.Sampler(N, D, dtype=torch.float32, seed=2, target="logistic", X=X, y=y,
                    flags=nat.FLAG_LOGISTIC_CUDA_CORES)
    xa, lpa = [host(t) for t in a.current()]
    xb, lpb = [host(t) for t in b.current()]
    assert np.array_equal(xa, xb)
    assert np.all(np.abs(lpa - lpb) <= 2e-5 * (1 + np.abs(lpb)))


def test_tc_run_is_sane(nat):
    """K = 5 iterations with resampling by N_eff: no device error, finite
    statistics, N_eff within (0, N]."""
    N, D, M, K = 8192, 32, 2048, 5
    X, y, _ = inputs.logistic_data(M, D, seed=6)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=4, target="logistic", X=X, y=y, step=0.05, init_scale=0.5)
    r = S.step(K, trace=True)
    S.sync()
    tr = nat.trace_dicts(r["trace"])
    for rec in tr:
        assert np.isfinite(rec["lse"]) and 0 < rec["ess"] <= N
    assert np.all(np.isfinite(host(r["mean"])))


def test_tc_timeout_is_reported_and_the_context_survives(nat):
    """Failure path without a GPU fault: with the test hook the likelihood's
    data copies are never issued, its bounded waits run out (~1 s), it
    drains and frees its tensor memory, and smc_sync reports SMC_ETIMEOUT.
    A normal sampler then runs on the same context."""
    X, y, _ = inputs.logistic_data(300, 8, seed=2)
    S = nat.Sampler(1000, 8, dtype=torch.float32, seed=1, target="logistic", X=X, y=y,
                    flags=nat.FLAG_TEST_STALL_LIKELIHOOD)
    with pytest.raises(nat.SmcError) as e:
        S.sync()
    assert e.value.code == nat.SMC_ETIMEOUT
    S.close()
    T = nat.Sampler(1000, 8, dtype=torch.float32, seed=1, target="logistic", X=X, y=y)
    r = T.step(2)
    T.sync()
    assert np.all(np.isfinite(host(r["mean"])))


def test_tc_full_size_sampled(nat, orc):
    """The logistic workload at full size, as the benchmark launches it:
    N = 2^18 particles, M = 8192 rows, D = 32, q_0 = N(0, 4I), step 0.5,
    iterations replayed from the CUDA graph.  The log-targets of 512 sampled
    particles (after the moves and resampling) against the oracle's, each
    computed one by one; the log-weights follow eq. (5) or the reset."""
    N, D, M, K = 1 << 18, 32, 8192, 3
    X, y, _ = inputs.logistic_data(M, D, seed=0)
    tgt = orc.Target.logistic(X.astype(np.float64), y.astype(np.float64), 4.0)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=11, target="logistic", X=X, y=y, prior_var=4.0, step=0.5,
                    init_scale=2.0)
    r = S.step(K, trace=True)
    S.sync()
    x, lp = [host(t) for t in S.current()]
    idx = np.random.default_rng(3).choice(N, size=512, replace=False)
    ref = tgt.logpi(x[idx].astype(np.float64))
    err = np.abs(lp[idx] - ref)
    assert np.all(err <= 2e-5 * (1 + np.abs(ref))), err.max()
    tr = nat.trace_dicts(r["trace"])
    assert [t["t"] for t in tr] == [1, 2, 3]
    lw = host(S.logw)
    if tr[-1]["resampled"]:
        assert np.all(lw == lw[0]) and abs(lw[0] + np.log(N)) < 1e-12 * np.log(N)
    assert np.all(np.isfinite(lw))
    print(f"full size: max |d log pi| over 512 particles = {err.max():.3e} (|log pi| up to {np.abs(ref).max():.0f})")


@pytest.mark.parametrize("warm,step", [(0, 0.5), (30, 0.05)])
def test_tc_weights_and_resampling_against_fp64(nat, orc, warm, step):
    """Reduced precision as resampling sees it (eq. (5), then Algorithm 4):
    N = 2^16 particles, M = 8192 rows, D = 32, q_0 = N(0, 4I).  warm = 0:
    the benchmark's step 0.5 from the initial draw; warm = 30: after 30
    resampling iterations with step 0.05 (a settled cloud whose weights are
    far less degenerate).  After one move and reweight, every particle's
    log w from the tensor-core likelihood is compared with the FP64 log w of
    the same particles (the oracle's log pi; log q_0 = -|x|^2 / 8 with
    constants dropped, Algorithm 2 line 1), bounded per particle by the
    arithmetic: the hi / lo split drops lo x lo (2^-18 of each product) and
    rounds each operand's lo part (2^-18), and FP32 accumulation adds ~2^-24
    per term, so |dz_m| <= 2^-16 sum_k |x_mk b_k| with margin; the epilogue's ex2 / lg2 add ~1e-7 per row; and
    eq. (5) takes the difference of the two FP32 log pi values (half an FP32
    ulp of the larger).  Then both weight vectors are resampled with the
    same Philox draw, and the share of particles whose copy counts differ is
    reported (printed with -s)."""
    N, D, M = 1 << 16, 32, 8192
    X, y, _ = inputs.logistic_data(M, D, seed=0)
    Xd = X.astype(np.float64)
    tgt = orc.Target.logistic(Xd, y.astype(np.float64), 4.0)
    seed = 7
    S = nat.Sampler(N, D, dtype=torch.float32, seed=seed, target="logistic", X=X, y=y, prior_var=4.0, step=step,
                    init_scale=2.0, resample_mode=nat.RESAMPLE_ALWAYS if warm else nat.RESAMPLE_NEVER)
    if warm:
        S.step(warm)
    x0, lp0 = [host(t).copy() for t in S.current()]
    lw0 = host(S.logw).copy()
    S.move()
    S.reweight()
    x1, lp1 = [host(t).copy() for t in S.current()]
    lw1 = host(S.logw).copy()
    S.sync()
    x0d, x1d = x0.astype(np.float64), x1.astype(np.float64)
    lp0_ref, lp1_ref = tgt.logpi(x0d), tgt.logpi(x1d)
    if warm:
        # the last warm-up iteration resampled: every log w is -log N
        assert np.all(lw0 == orc.reset_logw(N))
        lw0_ref = lw0
    else:
        q0 = -0.125 * np.sum(x0d * x0d, axis=1)
        # the sampler's initial weights are log pi - log q_0 with this q_0
        # (its log q_0 is formed in FP32)
        assert np.all(np.abs((lw0 - lp0.astype(np.float64)) + q0) <= 1e-6 * (1 + np.abs(q0)))
        lw0_ref = lp0_ref - q0
    lw1_ref = lw0_ref + (lp1_ref - lp0_ref)
    err = np.abs(lw1 - lw1_ref)
    # per-particle bound from the arithmetic
    abs_z = np.zeros(N)
    absX = np.abs(Xd)
    for a in range(0, N, 4096):
        abs_z[a:a + 4096] = (absX @ np.abs(x0d[a:a + 4096]).T).sum(axis=0) + (absX @ np.abs(x1d[a:a + 4096]).T).sum(axis=0)
    half_ulp = 0.5 * np.spacing(np.maximum(np.abs(lp0), np.abs(lp1)).astype(np.float32)).astype(np.float64)
    bound = 2.0 ** -16 * abs_z + 2e-6 * M + half_ulp
    assert np.all(err <= bound), (err.max(), float(np.argmax(err - bound)))
    # resampling both weight vectors with the same draw (seed, t = 1)
    nc_gpu, _ = nat.smc_resample_raw(torch.as_tensor(lw1, device="cuda"), seed, 1, nat.RESAMPLE_ALWAYS)
    nc_gpu = host(nc_gpu)
    nc_ref = orc.resample(lw1_ref, seed, 1, orc.RESAMPLE_ALWAYS)["ncopies"]
    assert nc_gpu.sum() == N and nc_ref.sum() == N
    differ = float(np.mean(nc_gpu != nc_ref))
    tv = 0.5 * float(np.abs(nc_gpu.astype(np.int64) - nc_ref).sum()) / N
    _, _, ess = orc.lse_ess(lw1_ref)
    q = np.quantile(err, [0.5, 0.9, 0.99, 1.0])
    print(f"\nwarm={warm} step={step}: |d log w| quantiles 50/90/99/100% = {q[0]:.3e} {q[1]:.3e} {q[2]:.3e} "
          f"{q[3]:.3e}; max err/bound {float((err / bound).max()):.3f}; |log pi| up to {np.abs(lp1_ref).max():.0f}; "
          f"N_eff (FP64) = {ess:.2f}; copy counts differ for {differ:.6f} of the particles "
          f"(total-variation distance of ncopies / N = {tv:.6f}); survivors GPU {np.count_nonzero(nc_gpu)}, "
          f"FP64 {np.count_nonzero(nc_ref)}")
