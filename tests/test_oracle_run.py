"""End-to-end pins of the oracle's Algorithm 2 loop against the closed form of
a Gaussian target: its posterior mean is mu and covariance Sigma.

The sampler's Monte Carlo error is not the ESS formula's (the forward-proposal
L-kernel of Sec. 5.2.3 leaves correlated, path-dependent weights), so the error
bar is measured from independent replicates: over R seeds the average estimate
must lie within 4.5 standard errors (across-seed std / sqrt(R)) of the truth.
A dropped term, a wrong sign or a transposed factor moves the average by many
standard errors.
"""
import math

import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs


def _replicates(orc, D, N, K, R, **kw):
    mu, Sigma = inputs.gaussian_target(D, seed=0)  # the C0 recipe
    tgt = orc.Target.gauss(mu, Sigma)
    fK, fhat, covs = [], [], []
    for seed in range(R):
        r = orc.run(tgt, N, seed, K, **kw)
        fK.append(r["means"][-1])
        fhat.append(r["fhat"])
        covs.append(np.diag(r["cov"]))
    return mu, Sigma, np.array(fK), np.array(fhat), np.array(covs)


def _within(est, truth, k=4.5):
    R = est.shape[0]
    se = est.std(axis=0, ddof=1) / math.sqrt(R)
    z = (est.mean(axis=0) - truth) / se
    assert np.all(np.abs(z) < k), z


def test_gaussian_posterior_moments_C0_shape(orc):
    # the plain FP64 sampler's shape (D=4, K=20, step 0.5, q0 = N(0, 4I)) at
    # N=8192 so the self-normalisation bias is well below the error bar
    mu, Sigma, fK, fhat, covs = _replicates(orc, D=4, N=8192, K=20, R=32)
    _within(fK, mu)
    _within(fhat, mu)          # eq. (6) recycled estimate
    # after 20 iterations the weighted covariance carries a finite-N bias that
    # shrinks with N (measured: -12% at N=2048, -7% at 8192, -4% at 65536; the
    # genealogy of the forward-kernel sampler coalesces); bound it loosely here
    # and test unbiasedness where the bias is negligible (K=2) below
    assert np.all(np.abs(covs.mean(axis=0) / np.diag(Sigma) - 1) < 0.2)
    mu, Sigma, fK2, _, covs2 = _replicates(orc, D=4, N=8192, K=2, R=32)
    _within(fK2, mu)
    _within(covs2, np.diag(Sigma))


def test_gaussian_posterior_moments_matched_start(orc):
    # q0 = N(0, I) on a standard-normal-like target: healthy ESS throughout, so
    # the error also shrinks like 1/sqrt(N) -- compare two sizes
    D = 2
    tgt = orc.Target.gauss(np.zeros(D), np.eye(D))
    errs = {}
    for N in (512, 8192):
        est = np.array([orc.run(tgt, N, s, 10, init_scale=1.0)["means"][-1] for s in range(24)])
        _within(est, np.zeros(D))
        errs[N] = np.sqrt(np.mean(est ** 2))
    assert errs[8192] < errs[512] / 2.0  # ~1/4 expected


def test_run_invariants(orc):
    mu, Sigma = inputs.gaussian_target(4, seed=0)
    tgt = orc.Target.gauss(mu, Sigma)
    N = 1024
    r = orc.run(tgt, N, 7, 20, ncopies_trace=True)
    tr = r["trace"]
    nct = r["ncopies"]
    for t in range(20):
        if tr[t, 4]:
            assert nct[t].sum() == N                          # eq. (9)
            assert tr[t, 5] == np.count_nonzero(nct[t])
            assert tr[t, 2] < N / 2                           # N_eff < N*
            if t + 1 < 20:
                assert abs(tr[t + 1, 1] - tr[t + 1, 0]) < 1e-12  # log c = LSE - 0
        else:
            assert not nct[t].any()
            assert tr[t, 2] >= N / 2 - 1e-6 * N
    if tr[-1, 4]:
        assert np.all(r["logw"] == -math.log(N))             # reset to 1/N
    # always-resample mode (the paper's worst case) resamples every iteration
    r2 = orc.run(tgt, N, 7, 5, mode=orc.RESAMPLE_ALWAYS)
    assert np.all(r2["trace"][:, 4] == 1)
    r3 = orc.run(tgt, N, 7, 5, mode=orc.RESAMPLE_NEVER)
    assert np.all(r3["trace"][:, 4] == 0)
    # t = 1 log c_t telescopes with the initial LSE on a no-resample run
    lse = r3["trace"][:, 0]
    np.testing.assert_allclose(np.cumsum(r3["trace"][:, 1])[1:], (lse - lse[0] + r3["trace"][0, 1])[1:],
                               atol=1e-9)


def test_run_deterministic(orc):
    mu, Sigma = inputs.gaussian_target(4, seed=0)
    tgt = orc.Target.gauss(mu, Sigma)
    a = orc.run(tgt, 300, 3, 6)
    b = orc.run(tgt, 300, 3, 6)
    np.testing.assert_array_equal(a["x"], b["x"])
    c = orc.run(tgt, 300, 4, 6)
    assert not np.array_equal(a["x"], c["x"])
