"""Pins of the oracle's deterministic elementary functions and of the
fixed-point exponential that quantises the weights, against high-precision
references (mpmath, decimal) and exact integer arithmetic."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest


def ulp(x):
    return math.ulp(abs(x)) if x != 0 else math.ulp(0.0)


def test_log_within_two_ulp(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    g = np.random.default_rng(0)
    pts = list(g.uniform(0, 1, 3000)) + list(2.0 ** g.uniform(-53, 0, 2000)) + [
        1.0, 0.5, 2.0, 2 ** -53, 1 - 2 ** -53, 1024.0, float(2 ** 24), float(2 ** 31), 3.0, 1e-300]
    pts += list(g.uniform(1, 2 ** 31, 500))
    for u in pts:
        if u <= 0:
            continue
        got = orc.det_log(u)
        ref = float(mp.log(mp.mpf(u)))
        assert abs(got - ref) <= 2 * ulp(ref) + 1e-300, (u, got, ref)


def test_sincos2pi_within_two_ulp(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    g = np.random.default_rng(1)
    vs = [int(v) for v in g.integers(0, 2 ** 53, 4000, dtype=np.uint64)]
    vs += [0, 1, 2 ** 50, 2 ** 51, 2 ** 52, 3 * 2 ** 51, 2 ** 53 - 1, 2 ** 50 - 1, 2 ** 50 + 1]
    for v in vs:
        a = mp.mpf(v) / mp.mpf(2) ** 53
        s, c = orc.det_sincos2pi_u53(v)
        rs, rc = float(mp.sinpi(2 * a)), float(mp.cospi(2 * a))
        # absolute bound near zeros of sin/cos, relative elsewhere
        assert abs(s - rs) <= 2 * ulp(rs) + 2 ** -54, (v, s, rs)
        assert abs(c - rc) <= 2 * ulp(rc) + 2 ** -54, (v, c, rc)


def _exact_E(y):
    getcontext().prec = 60
    return Decimal(2) ** 62 * Decimal(y).exp()


def test_expfx_against_decimal(orc):
    g = np.random.default_rng(2)
    ys = list(-g.uniform(0, 44, 4000)) + list(-g.exponential(1e-3, 500)) + [
        0.0, -0.0, -1e-300, -2 ** -60, -1.0, -math.log(2), -43.9, -43.5, -10.0, -27.0]
    worst = 0.0
    for y in ys:
        E = orc.expfx(y)
        X = _exact_E(y)
        err = abs(Decimal(E) - X)
        # relative error 2^-54 of the exact value plus one unit of truncation
        bound = X * Decimal(2) ** -54 + 1
        assert err <= bound, (y, E, X)
        if X > 2 ** 58:
            worst = max(worst, float(err / X))
    assert worst < 2 ** -54


def test_expfx_special_values(orc):
    assert orc.expfx(0.0) == 2 ** 62
    assert orc.expfx(-0.0) == 2 ** 62
    assert orc.expfx(-math.inf) == 0
    assert orc.expfx(-44.0) == 0
    assert orc.expfx(-1000.0) == 0
    # non-decreasing in y up to the few units of table/Horner rounding
    ys = np.sort(-np.random.default_rng(3).uniform(0, 44, 3000))
    Es = [orc.expfx(float(y)) for y in ys]
    assert all(b >= a - 64 for a, b in zip(Es, Es[1:]))


def test_expfx_table_exact_roots(orc):
    # T1[j] ~ 2^63 2^(-j/64), T2[j] ~ 2^63 2^(-j/4096); built from integer
    # square roots, so within a few units of the exactly rounded value
    getcontext().prec = 60
    T = orc.expfx_table()
    assert int(T[0]) == 2 ** 63 and int(T[64]) == 2 ** 63
    for j in range(64):
        exact1 = Decimal(2) ** 63 * (Decimal(2) ** (Decimal(-j) / 64))
        exact2 = Decimal(2) ** 63 * (Decimal(2) ** (Decimal(-j) / 4096))
        assert abs(Decimal(int(T[j])) - exact1) <= 16, j
        assert abs(Decimal(int(T[64 + j])) - exact2) <= 32, j
    # T1[32] = floor(2^63 / sqrt 2) = isqrt(2^125) exactly (one square-root step)
    assert int(T[32]) == math.isqrt(2 ** 125)
    # the c_b chain continued six more times: T2[32] = isqrt applied to T1[1]
    assert int(T[64 + 32]) == math.isqrt(int(T[1]) << 63)


def test_quant_shift(orc):
    assert orc.quant_shift(1) == 62
    assert orc.quant_shift(2) == 62
    assert orc.quant_shift(3) == 61
    assert orc.quant_shift(1024) == 53
    assert orc.quant_shift(1025) == 52
    assert orc.quant_shift(2 ** 24) == 39
    assert orc.quant_shift(2 ** 24 + 1) == 38
    for N in (1, 7, 1000, 2 ** 20, 2 ** 24, 2 ** 30):
        F = orc.quant_shift(N)
        assert N * 2 ** F <= 2 ** 63  # S cannot overflow 64 bits
        assert N * N * 2 ** (2 * F) < 2 ** 127  # N sum W^2 fits 128 bits


def test_reset_logw(orc):
    for N in (1, 2, 1000, 1024, 2 ** 24, 3 * 2 ** 20):
        assert abs(orc.reset_logw(N) + math.log(N)) <= 2 * ulp(math.log(N)) + 1e-300
