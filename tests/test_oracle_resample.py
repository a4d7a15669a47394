"""Pins of systematic resampling (MVR) and of Sequential Redistribute.

MVR is only named in the paper (Sec. 3.3, Algorithm 4); the reading used is
systematic resampling on the integer CDF of the quantised weights.  Its pins
are eq. (9) (sum ncopies = N), the floor bounds of systematic resampling, its
unbiasedness checked exhaustively over every offset U for small S, and
hand-worked examples.  S-R (Algorithm 5) is pinned by brute force over all
compositions of small N.
"""
import itertools
import os

import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ints(s):
    return [int(v) for v in s.split(",")]


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [p.strip() for p in line.split("|")]


def test_systematic_golden(orc):
    for N, W, U, nc, off in _golden("systematic_small.txt"):
        W = np.array(_ints(W), dtype=np.uint64)
        got_nc, got_off = orc.systematic(W, int(W.sum()), int(U))
        assert len(W) == int(N)
        assert list(got_nc) == _ints(nc)
        assert list(got_off) == _ints(off)


def test_redistribute_golden(orc):
    for nc, rows, out in _golden("sr_small.txt"):
        x = np.array([ord(r) for r in rows.split(",")], dtype=np.int64)[:, None]
        got = orc.redistribute(np.array(_ints(nc), dtype=np.int32), x)
        assert [chr(int(v)) for v in got[:, 0]] == out.split(",")


@pytest.mark.parametrize("seed", range(20))
def test_systematic_invariants(orc, seed):
    g = np.random.default_rng(seed)
    N = int(g.integers(1, 3000))
    W = g.integers(0, 2 ** 30, size=N, dtype=np.uint64)
    if seed % 3 == 0:
        W[g.uniform(size=N) < 0.7] = 0
    if W.sum() == 0:
        W[0] = 1
    S = int(W.sum())
    U = int(g.integers(0, S))
    nc, off = orc.systematic(W, S, U)
    assert nc.sum() == N  # eq. (9)
    lo = (N * W.astype(object)) // S
    assert np.all(nc >= lo) and np.all(nc <= lo + 1)
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(nc)[:-1]]).astype(np.uint32))


@pytest.mark.parametrize("seed", range(12))
def test_systematic_unbiased_exhaustive(orc, seed):
    # E_U[ncopies_i] = N W_i / S, checked exactly by summing over all U in [0, S)
    g = np.random.default_rng(100 + seed)
    N = int(g.integers(1, 9))
    W = g.integers(0, 9, size=N, dtype=np.uint64)
    if W.sum() == 0:
        W[-1] = 3
    S = int(W.sum())
    tot = np.zeros(N, dtype=np.int64)
    for U in range(S):
        nc, _ = orc.systematic(W, S, U)
        assert nc.sum() == N
        tot += nc
    np.testing.assert_array_equal(tot, N * W.astype(np.int64))


def test_systematic_one_hot_and_equal(orc):
    for N in (1, 2, 5, 1000):
        for j in {0, N // 2, N - 1}:
            W = np.zeros(N, dtype=np.uint64)
            W[j] = 12345
            for U in (0, 1, 12344):
                nc, _ = orc.systematic(W, 12345, U)
                e = np.zeros(N, dtype=np.int32)
                e[j] = N
                np.testing.assert_array_equal(nc, e)
        W = np.full(N, 2 ** 20, dtype=np.uint64)
        for U in (0, 7, N * 2 ** 20 - 1):
            nc, _ = orc.systematic(W, N * 2 ** 20, U)
            np.testing.assert_array_equal(nc, np.ones(N, dtype=np.int32))


def test_decision_rule(orc):
    # strict N_eff < N/2 (Sec. 3.1, Algorithm 2), on the quantised weights
    assert not orc.decide(4, 2, 2)     # W=[1,1,0,0]: N_eff = 2 = N/2
    assert not orc.decide(4, 4, 6)     # W=[2,1,1,0]: N_eff = 8/3
    assert orc.decide(4, 4, 10)        # W=[3,1,0,0]: N_eff = 1.6
    assert orc.decide(3, 10, 68)       # odd N: N_eff = 100/68 < 1.5
    assert not orc.decide(3, 10, 66)   # N_eff = 100/66 > 1.5
    assert orc.decide(4, 2, 2, orc.RESAMPLE_ALWAYS)
    assert not orc.decide(4, 4, 10, orc.RESAMPLE_NEVER)
    g = np.random.default_rng(5)
    for _ in range(300):
        N = int(g.integers(2, 500))
        W = g.integers(0, 2 ** 20, size=N).astype(np.int64) ** int(g.integers(1, 4))
        W = np.minimum(W, 2 ** 30).astype(np.uint64)
        if W.sum() == 0:
            continue
        S = int(W.sum())
        s2 = int((W.astype(object) ** 2).sum())
        ess = S * S / s2
        if abs(ess - N / 2) > 1e-9 * N:
            assert orc.decide(N, S, s2) == (ess < N / 2)


def test_resample_on_logw_special_cases(orc):
    N = 777
    r = orc.resample(np.zeros(N), seed=1, t=1, mode=orc.RESAMPLE_ALWAYS)
    np.testing.assert_array_equal(r["ncopies"], np.ones(N, dtype=np.int32))
    assert not orc.resample(np.full(N, -3.5), 1, 1)["did"]  # N_eff = N
    lw = np.full(N, -np.inf)
    lw[123] = 4.0
    r = orc.resample(lw, 1, 1)
    assert r["did"] and r["ncopies"][123] == N and r["ncopies"].sum() == N
    with pytest.raises(FloatingPointError):
        orc.resample(np.full(N, -np.inf), 1, 1)
    bad = np.zeros(N)
    bad[5] = np.nan
    with pytest.raises(FloatingPointError):
        orc.resample(bad, 1, 1)


def test_resample_quantisation_consistent(orc):
    g = np.random.default_rng(11)
    for s in (0.5, 2.0, 8.0):
        lw = g.normal(0, s, size=5000)
        r = orc.resample(lw, seed=2, t=3, mode=orc.RESAMPLE_ALWAYS)
        F = orc.quant_shift(lw.size)
        m = lw.max()
        W = np.array([orc.expfx(v - m) >> (62 - F) for v in lw], dtype=np.uint64)
        np.testing.assert_array_equal(r["W"], W)
        assert r["S"] == int(W.astype(object).sum())
        assert r["ncopies"].sum() == lw.size
        # copies follow the normalised weights: |ncopies - N w~| < 1 + N 2^-F
        w = np.exp(lw - m)
        w /= w.sum()
        assert np.max(np.abs(r["ncopies"] - lw.size * w)) < 1 + 1e-6


@pytest.mark.parametrize("N", range(1, 7))
def test_redistribute_all_compositions(orc, N):
    # every ncopies vector with sum N (eq. (9)): output is the stable repeat
    x = (np.arange(N * 3, dtype=np.float64).reshape(N, 3) + 0.25)
    for cut in itertools.combinations_with_replacement(range(N), N):
        nc = np.bincount(np.array(cut), minlength=N).astype(np.int32)
        out = orc.redistribute(nc, x)
        ref = np.repeat(x, nc, axis=0)
        np.testing.assert_array_equal(out, ref)


def test_redistribute_bytes_any_dtype(orc):
    g = np.random.default_rng(0)
    for dt, D in ((np.float32, 16), (np.float32, 3), (np.float64, 4), (np.uint8, 5)):
        N = 1000
        x = (g.standard_normal((N, D)) * 100).astype(dt)
        nc = np.bincount(g.integers(0, N, N), minlength=N).astype(np.int32)
        np.testing.assert_array_equal(orc.redistribute(nc, x), np.repeat(x, nc, axis=0))


def test_decide_threshold_against_exact_rationals(orc):
    """Algorithm 2, line 7 with a general N*: resample iff N_eff < N*, where
    N_eff = S^2 / sum W^2 (eq. (1) on the quantised weights), compared with
    exact rational arithmetic; nstar = 0 is the paper's N* = N/2."""
    from fractions import Fraction

    g = np.random.default_rng(11)
    for trial in range(300):
        N = int(g.integers(1, 40))
        W = [int(v) for v in g.integers(0, 2 ** 20, size=N)]
        if trial % 5 == 0:
            W = [w if g.uniform() < 0.3 else 0 for w in W]
        if sum(W) == 0:
            W[0] = 1
        S, S2 = sum(W), sum(w * w for w in W)
        neff = Fraction(S * S, S2)
        assert orc.decide(N, S, S2, nstar=0) == (neff < Fraction(N, 2)), (W,)
        for nstar in range(1, N + 1):
            assert orc.decide(N, S, S2, nstar=nstar) == (neff < nstar), (W, nstar)


def test_decide_threshold_closed_forms(orc):
    # equal weights: N_eff = N, never below N* <= N; one-hot: N_eff = 1
    for N in (1, 2, 7, 1000):
        for nstar in (1, max(1, N // 2), N):
            assert not orc.decide(N, N * 5, N * 25, nstar=nstar)
            assert orc.decide(N, 9, 81, nstar=nstar) == (nstar > 1)
    # the modes override the threshold
    assert orc.decide(10, 9, 81, mode=orc.RESAMPLE_NEVER, nstar=10) is False
    assert orc.decide(10, 50, 250, mode=orc.RESAMPLE_ALWAYS, nstar=1) is True


def test_run_threshold_extremes_match_the_modes(orc):
    """N* = 1 never resamples (N_eff >= 1 always) and N* = N resamples unless
    every weight is equal: whole runs equal the NEVER and ALWAYS runs."""
    mu, Sigma = inputs.gaussian_target(3, seed=2)
    tgt = orc.Target.gauss(mu, Sigma)
    N, K = 500, 5
    never = orc.run(tgt, N, 4, K, mode=orc.RESAMPLE_NEVER)
    always = orc.run(tgt, N, 4, K, mode=orc.RESAMPLE_ALWAYS)
    low = orc.run(tgt, N, 4, K, nstar=1)
    high = orc.run(tgt, N, 4, K, nstar=N)
    for a, b in ((low, never), (high, always)):
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["logw"], b["logw"])
        assert np.array_equal(a["trace"], b["trace"])
    # a threshold between gives a decision sequence between the two
    mid = orc.run(tgt, N, 4, K, nstar=N // 4)
    assert set(mid["trace"][:, 4]) <= {0.0, 1.0}
