"""The Student-t target of Sec. 5.2.3 (D = 1, eq. (14)) over whole runs.

FP64: the moves are bit-identical to the oracle's (same Philox draws, same
explicitly rounded operations); log pi differs from the oracle's only through
CUDA's log1p against glibc's (<= a few ulp), so log pi and log w agree within
1e-12 relative and the copy counts of every iteration -- integers from the
quantised weights -- and hence the particles agree exactly.  Both precisions
also recover the target's closed-form moments (mean mu, variance
nu / (nu - 2)) within Monte Carlo error across independent runs, also for the
recycled estimate of eq. (6).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10252_gb300 import build, native

    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    native.lib()
    return native


def test_student_fp64_run_matches_oracle(nat, orc):
    N, K, mu, nu = 4000, 6, 1.5, 5.0
    tgt = orc.Target.student_t(mu, nu)
    S = nat.Sampler(N, 1, dtype=torch.float64, seed=8, target="student_t", mu=[mu], nu=nu, step=0.8,
                    init_scale=2.0)
    r = S.step(K, trace=True)
    ref = orc.run(tgt, N, 8, K, init_scale=2.0, step=0.8)
    S.sync()
    tr = nat.trace_dicts(r["trace"])
    for k in range(K):
        assert tr[k]["resampled"] == int(ref["trace"][k][4])
        assert abs(tr[k]["lse"] - ref["trace"][k][0]) <= 1e-10 * (1 + abs(ref["trace"][k][0]))
    x, lp = [t.cpu().numpy() for t in S.current()]
    assert np.array_equal(x, ref["x"])
    assert np.all(np.abs(lp - ref["logpi"]) <= 1e-12 * (1 + np.abs(ref["logpi"])))
    lw = S.logw.cpu().numpy()
    assert np.all(np.abs(lw - ref["logw"]) <= 1e-12 * (1 + np.abs(ref["logw"])))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_student_posterior_moments(nat, dtype):
    """E[x] = mu and Var[x] = nu / (nu - 2): the estimates of 16 independent
    runs (seeds), averaged, within 4.5 standard errors taken across the runs
    (a single run's error is dominated by resampling and correlated moves,
    which an i.i.d. bound does not describe)."""
    N, K, mu, nu, R = 1 << 15, 30, -0.7, 6.0, 16
    var = nu / (nu - 2.0)
    means, covs, fhats = [], [], []
    for seed in range(R):
        S = nat.Sampler(N, 1, dtype=dtype, seed=100 + seed, target="student_t", mu=[mu], nu=nu, step=1.0,
                        init_scale=3.0)
        r = S.step(K, cov=True, fhat=True)
        S.sync()
        means.append(float(r["mean"].cpu()[0]))
        covs.append(float(r["cov"].cpu()[0, 0]))
        fhats.append(float(r["fhat"].cpu()[0]))
        S.close()
    for vals, target in ((means, mu), (fhats, mu), (covs, var)):
        v = np.asarray(vals)
        se = v.std(ddof=1) / np.sqrt(R)
        assert abs(v.mean() - target) <= 4.5 * se + 1e-12, (v.mean(), target, se)


def test_student_fp32_logpi_against_oracle(nat, orc):
    """FP32 Student-t log pi (eq. (14)) of the initial and moved particles
    against the oracle's FP64 values, within the reduced-precision bound."""
    N, mu, nu = 50001, -0.3, 4.0
    tgt = orc.Target.student_t(mu, nu)
    S = nat.Sampler(N, 1, dtype=torch.float32, seed=12, target="student_t", mu=[mu], nu=nu, step=0.7,
                    init_scale=2.0, resample_mode=nat.RESAMPLE_NEVER)
    for _ in range(2):
        x, lp = [t.cpu().numpy().copy() for t in S.current()]
        ref = tgt.logpi(x.astype(np.float64))
        assert np.all(np.abs(lp - ref) <= 2e-5 * (1 + np.abs(ref))), np.abs(lp - ref).max()
        S.move()
        S.reweight()
    S.sync()
