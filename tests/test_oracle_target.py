"""Pins of the oracle's targets and of eqs. (1), (2), (5), (7) against textbook
routines (numpy.linalg, scipy.special/stats) and closed forms."""
import math

import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs


@pytest.mark.parametrize("D", [1, 2, 4, 16, 32])
def test_cholesky_and_gauss_logpi(orc, D):
    mu, Sigma = inputs.gaussian_target(D, seed=D)
    L = orc.cholesky(Sigma)
    np.testing.assert_allclose(L, np.linalg.cholesky(Sigma), rtol=1e-12, atol=1e-12)
    tgt = orc.Target.gauss(mu, Sigma)
    x = np.random.default_rng(D).standard_normal((50, D)) * 3
    got = tgt.logpi(x)
    P = np.linalg.inv(Sigma)
    d = x - mu
    ref = -0.5 * np.einsum("ni,ij,nj->n", d, P, d)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)
    assert tgt.logpi(mu[None])[0] == 0.0


def test_cholesky_rejects_indefinite(orc):
    with pytest.raises(ValueError):
        orc.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_logistic_logpi_naive(orc):
    X, y, beta = inputs.logistic_data(64, 5, seed=3)
    tgt = orc.Target.logistic(X.astype(np.float64), y.astype(np.float64), 4.0)
    B = np.random.default_rng(0).standard_normal((20, 5))
    got = tgt.logpi(B)
    ref = []
    for b in B:
        s = 0.0
        for m in range(64):
            z = sum(float(X[m, c]) * b[c] for c in range(5))
            s += float(y[m]) * z - math.log1p(math.exp(z))
        ref.append(s - float(b @ b) / 8.0)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-10)


def _logistic_target(orc, M=200, D=6, seed=4, prior_var=4.0):
    X, y, _ = inputs.logistic_data(M, D, seed=seed)
    return X.astype(np.float64), y.astype(np.float64), orc.Target.logistic(X.astype(np.float64),
                                                                          y.astype(np.float64), prior_var)


def test_logistic_logpi_at_zero_is_minus_m_log2(orc):
    """b = 0: every z_m = 0 and each row contributes -log 2 whatever its label."""
    X, y, tgt = _logistic_target(orc)
    got = tgt.logpi(np.zeros((1, X.shape[1])))[0]
    assert abs(got - (-X.shape[0] * math.log(2.0))) <= 1e-12 * X.shape[0]


def test_logistic_logpi_is_bernoulli_loglik_plus_gaussian_prior(orc):
    """log pi = sum_m log Bernoulli(y_m | sigmoid(z_m)) + log N(b | 0, v I) up to
    the prior's constant: scipy's logistic log-probabilities (log_expit) and
    normal log-density, an implementation independent of the oracle."""
    sp = pytest.importorskip("scipy.special")
    ss = pytest.importorskip("scipy.stats")
    X, y, tgt = _logistic_target(orc, prior_var=2.5)
    B = np.random.default_rng(1).standard_normal((15, X.shape[1])) * 1.5
    got = tgt.logpi(B)
    D = X.shape[1]
    const = D * 0.5 * math.log(2.0 * math.pi * 2.5)
    for b, g in zip(B, got):
        z = X @ b
        ll = np.sum(y * sp.log_expit(z) + (1.0 - y) * sp.log_expit(-z))
        lp = np.sum(ss.norm.logpdf(b, scale=math.sqrt(2.5))) + const
        assert abs(g - (ll + lp)) <= 1e-9 * (1.0 + abs(g))


def test_logistic_logpi_gradient_matches_closed_form(orc):
    """Central differences of the oracle's log pi against the closed-form
    gradient X^T (y - sigmoid(X b)) - b / v (a dropped term, a wrong sign or a
    transposed X shows up here)."""
    X, y, tgt = _logistic_target(orc, M=120, D=5, prior_var=3.0)
    b = np.array([0.3, -0.7, 1.1, 0.05, -1.4])
    g = X.T @ (y - 1.0 / (1.0 + np.exp(-(X @ b)))) - b / 3.0
    h = 1e-5
    for c in range(5):
        e = np.zeros(5)
        e[c] = h
        fd = (tgt.logpi((b + e)[None])[0] - tgt.logpi((b - e)[None])[0]) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * (1.0 + abs(g[c]))


def test_logistic_logpi_label_flip_symmetry(orc):
    """sigmoid(-z) = 1 - sigmoid(z): flipping every label and negating b leaves
    the likelihood unchanged, and the prior is symmetric."""
    X, y, tgt = _logistic_target(orc)
    flip = orc.Target.logistic(X, 1.0 - y, 4.0)
    B = np.random.default_rng(2).standard_normal((10, X.shape[1]))
    np.testing.assert_allclose(tgt.logpi(B), flip.logpi(-B), rtol=1e-13, atol=1e-10)


def test_student_t_logpi(orc):
    st = pytest.importorskip("scipy.stats")
    tgt = orc.Target.student_t(1.5, 5.0)
    x = np.linspace(-20, 20, 81)[:, None]
    got = tgt.logpi(x)
    ref = st.t.logpdf(x[:, 0], df=5.0, loc=1.5)
    # unnormalised: equal up to the log normalising constant
    np.testing.assert_allclose(got - ref, np.full_like(got, (got - ref)[0]), atol=1e-12)


def test_lse_ess_closed_forms(orc):
    for N in (1, 2, 1000):
        m, lse, ess = orc.lse_ess(np.full(N, -2.0))
        assert ess == N
        assert abs(lse - (-2.0 + math.log(N))) < 1e-13
        lw = np.full(N, -np.inf)
        lw[N // 2] = 7.0
        m, lse, ess = orc.lse_ess(lw)
        assert ess == 1.0 and lse == 7.0 and m == 7.0
    with pytest.raises(FloatingPointError):
        orc.lse_ess(np.full(5, -np.inf))
    with pytest.raises(FloatingPointError):
        orc.lse_ess(np.array([0.0, np.nan]))


def test_lse_ess_against_scipy(orc):
    sp = pytest.importorskip("scipy.special")
    g = np.random.default_rng(1)
    for s in (0.5, 2, 8, 30):
        lw = g.normal(0, s, 4000)
        m, lse, ess = orc.lse_ess(lw)
        assert abs(lse - sp.logsumexp(lw)) < 1e-10
        w = sp.softmax(lw)
        assert abs(ess - 1.0 / np.sum(w * w)) < 1e-9 * ess  # eq. (1)


def test_estimate_against_numpy(orc):
    g = np.random.default_rng(2)
    x = g.standard_normal((3000, 4)) + 1
    lw = g.normal(0, 2, 3000)
    m, lse, ess = orc.lse_ess(lw)
    mean, cov = orc.estimate(x, lw, lse)
    w = np.exp(lw - lse)
    np.testing.assert_allclose(mean, np.average(x, axis=0, weights=w), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(cov, np.cov(x.T, aweights=w, bias=True), rtol=1e-9, atol=1e-11)


def test_reweight_forward_kernel_term_is_zero(orc):
    # eq. (5) with L = q (Sec. 5.2.3): the weight update is pi(x_t)/pi(x_{t-1})
    mu, Sigma = inputs.gaussian_target(3, 0)
    tgt = orc.Target.gauss(mu, Sigma)
    g = np.random.default_rng(4)
    xp = g.standard_normal((100, 3))
    x = xp + 0.5 * g.standard_normal((100, 3))
    lpp = tgt.logpi(xp)
    lw = g.normal(0, 1, 100)
    lw2, lp = orc.reweight(tgt, xp, x, lpp, lw, 0.5)
    np.testing.assert_array_equal(lp, tgt.logpi(x))
    np.testing.assert_array_equal(lw2, lw + (lp - lpp))


def test_init_weights_are_pi_over_q0(orc):
    # Algorithm 2 line 1: w0 = pi(x0)/q0(x0), q0 = N(0, s^2 I) (constants dropped)
    mu, Sigma = inputs.gaussian_target(4, 0)
    tgt = orc.Target.gauss(mu, Sigma)
    x, lw, lp = orc.init(tgt, 500, seed=3, init_scale=2.0)
    np.testing.assert_array_equal(lp, tgt.logpi(x))
    np.testing.assert_allclose(lw, lp + 0.5 * np.sum(x * x, axis=1) / 4.0, rtol=1e-13, atol=1e-12)
    assert abs(np.std(x) - 2.0) < 0.1
