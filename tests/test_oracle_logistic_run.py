"""Pin of the oracle's Algorithm 2 loop on the Bayesian logistic-regression
target against numerical quadrature of its posterior.

For D = 1 and D = 2 the posterior p(b | X, y) ~ exp(sum_m [y_m z_m -
log(1 + e^z_m)] - |b|^2 / (2 prior_var)), z = X b, is integrated on a fine
grid (an independent numpy evaluation of the density, trapezoidal weights),
which gives its mean and variances to far better than the sampler's Monte
Carlo error.  As in the Gaussian pins, the error bar comes from independent
replicates: over R seeds the average estimate f_K (eq. (7)) and the average
weighted variance must lie within 4.5 standard errors of the quadrature
values.  A wrong sign in the likelihood, a dropped prior term, a transposed
X or a mis-scaled proposal moves the average by many standard errors.
"""
import math

import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs

PRIOR_VAR = 4.0


def _log_post(B, X, y):
    # B: [G, D] grid points -> log density up to a constant
    Z = B @ X.T  # [G, M]
    ll = (y[None, :] * Z - np.logaddexp(0.0, Z)).sum(axis=1)
    return ll - (B * B).sum(axis=1) / (2.0 * PRIOR_VAR)


def _quadrature_moments(X, y):
    D = X.shape[1]
    if D == 1:
        g = np.linspace(-12.0, 12.0, 40001)
        B = g[:, None]
        lp = _log_post(B, X, y)
        w = np.exp(lp - lp.max())
        w[0] *= 0.5
        w[-1] *= 0.5
        mean = np.array([(w * g).sum() / w.sum()])
        var = np.array([(w * (g - mean[0]) ** 2).sum() / w.sum()])
        return mean, var
    g = np.linspace(-9.0, 9.0, 721)
    G0, G1 = np.meshgrid(g, g, indexing="ij")
    B = np.stack([G0.ravel(), G1.ravel()], axis=1)
    lp = _log_post(B, X, y)
    w = np.exp(lp - lp.max()).reshape(G0.shape)
    tw = np.ones_like(g)
    tw[0] = tw[-1] = 0.5
    w = w * tw[:, None] * tw[None, :]
    w = w.ravel()
    mean = (w[:, None] * B).sum(axis=0) / w.sum()
    var = (w[:, None] * (B - mean) ** 2).sum(axis=0) / w.sum()
    return mean, var


def _within(est, truth, k=4.5):
    R = est.shape[0]
    se = est.std(axis=0, ddof=1) / math.sqrt(R)
    z = (est.mean(axis=0) - truth) / se
    assert np.all(np.abs(z) < k), (z, est.mean(axis=0), truth)


@pytest.mark.parametrize("D,M", [(1, 40), (2, 60)])
def test_logistic_posterior_moments_against_quadrature(orc, D, M):
    X, y, _ = inputs.logistic_data(M, D, seed=11)
    X64, y64 = X.astype(np.float64), y.astype(np.float64)
    mean_q, var_q = _quadrature_moments(X64, y64)
    tgt = orc.Target.logistic(X64, y64, PRIOR_VAR)

    def replicates(N, K, R):
        fK, var = [], []
        for seed in range(R):
            r = orc.run(tgt, N, seed, K, init_scale=2.0, step=0.5)
            fK.append(r["means"][-1])
            var.append(np.diag(r["cov"]))
        return np.array(fK), np.array(var)

    # after 30 iterations: the mean within its error bar; the weighted
    # variance carries the finite-N bias of the coalescing genealogy (as for
    # the Gaussian target, a few per cent low at these N), bounded loosely
    fK, var = replicates(4096, 30, 12)
    _within(fK, mean_q)
    assert np.all(np.abs(var.mean(axis=0) / var_q - 1) < 0.2), (var.mean(axis=0), var_q)
    # after two iterations, where that bias is negligible: both moments within
    # their error bars
    fK2, var2 = replicates(8192, 2, 16)
    _within(fK2, mean_q)
    _within(var2, var_q)
    # the data are informative: the posterior is much narrower than the prior
    assert np.all(var_q < PRIOR_VAR / 2)


def test_logistic_quadrature_pins_itself():
    # the quadrature recipe reproduces a conjugate case exactly: with no data
    # rows the posterior is the prior N(0, PRIOR_VAR I)
    X = np.zeros((1, 2))
    y = np.zeros(1)
    # one row of zeros contributes the constant -log 2: the posterior is the prior
    mean, var = _quadrature_moments(X, y)
    np.testing.assert_allclose(mean, 0.0, atol=1e-9)
    np.testing.assert_allclose(var, PRIOR_VAR, rtol=2e-3)
    X1 = np.zeros((1, 1))
    mean1, var1 = _quadrature_moments(X1, y)
    np.testing.assert_allclose(mean1, 0.0, atol=1e-9)
    np.testing.assert_allclose(var1, PRIOR_VAR, rtol=1e-6)
