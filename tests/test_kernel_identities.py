"""Host checks of two identities the CUDA kernels rely on for exact results.

* The move kernel, when every log-weight started at the same value R (the
  iteration after a resampling), takes the block maximum of
  log w_i = R + double(dlt_i) on the FP32 differences dlt_i with 32-bit
  integer-ordered keys and converts once: R + double(max dlt).  That equals
  the maximum of the FP64 values because x -> R + double(x) never decreases
  (IEEE addition rounds monotonically), including -0 / +0 and infinities.
* The quantise scan computes off = floor((N C + U) / S) from the estimate
  mulhi(C, floor(N 2^64 / S)) and at most three exact corrections, which
  needs floor((N C + U) / S) - estimate <= 3 whenever C <= S, U < S and
  S >= 2^(63 - ceil(log2 N)) (the fixed-point scale of the weights).
"""
import math
import struct

import numpy as np
import pytest


def _key64(v: float) -> int:
    # integer-ordered key of a double (-0 below +0), as the kernels' ordered_key
    b = struct.unpack("<q", struct.pack("<d", v))[0]
    return b if b >= 0 else b ^ 0x7FFFFFFFFFFFFFFF


def _key32(f: np.float32) -> int:
    b = struct.unpack("<i", struct.pack("<f", float(f)))[0]
    return b if b >= 0 else b ^ 0x7FFFFFFF


def _from_key32(k: int) -> np.float32:
    b = k if k >= 0 else k ^ 0x7FFFFFFF
    return np.float32(struct.unpack("<f", struct.pack("<i", b))[0])


def _fp64_max(R: float, dlt: np.ndarray) -> float:
    vals = [R + float(d) for d in dlt]
    return max(vals, key=_key64)


def _fp32_route(R: float, dlt: np.ndarray) -> float:
    k = max(_key32(d) for d in dlt)
    return R + float(_from_key32(k))


SPECIAL = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 3.4e38, -3.4e38, 1.0, -1.0], dtype=np.float32)


@pytest.mark.parametrize("seed", range(8))
def test_fp32_difference_maximum_equals_fp64_maximum(seed):
    rng = np.random.default_rng(seed)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        scale = float(10.0 ** rng.integers(-8, 6))
        dlt = (rng.standard_normal(n) * scale).astype(np.float32)
        if trial % 3 == 0:  # mix in signed zeros, infinities, extremes
            dlt[rng.integers(0, n, size=max(1, n // 4))] = rng.choice(SPECIAL, size=max(1, n // 4))
        if trial % 5 == 0:  # ties and near-ties that round to the same double sum
            dlt[:] = dlt[0]
        R = float(rng.choice([-math.log(1 << int(rng.integers(0, 31))), -0.0, -17.25,
                              float(rng.standard_normal()) * 1e3]))
        a, b = _fp64_max(R, dlt), _fp32_route(R, dlt)
        assert _key64(a) == _key64(b), (R, dlt, a, b)


def test_signed_zero_cases():
    # R = -0.0 (one particle: -log 1): -0 + -0 = -0 and -0 + +0 = +0
    for dlt in ([-0.0], [0.0], [-0.0, 0.0], [0.0, -0.0]):
        d = np.array(dlt, dtype=np.float32)
        assert _key64(_fp64_max(-0.0, d)) == _key64(_fp32_route(-0.0, d))


def _ceil_log2(n: int) -> int:
    return (n - 1).bit_length()


def _offset_estimate_gap(n: int, S: int, U: int, C: int) -> int:
    R = (n << 64) // S
    est = (C * R) >> 64
    exact = (n * C + U) // S
    return exact - est


@pytest.mark.parametrize("seed", range(6))
def test_scan_quotient_needs_at_most_three_corrections(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(3000):
        n = int(rng.integers(1, 1 << 31))
        F = min(62, 63 - _ceil_log2(n))
        lo = 1 << F
        # S from the smallest admissible sum up to N * 2^F (every weight at its largest)
        S = int(rng.integers(lo, max(lo + 1, min(n * (1 << F), (1 << 63) - 1))))
        U = int(rng.integers(0, S))
        C = int(rng.integers(0, S + 1))
        gap = _offset_estimate_gap(n, S, U, C)
        assert 0 <= gap <= 3, (n, S, U, C, gap)


def test_scan_quotient_edges():
    for n in (1, 2, 3, 1000, (1 << 24) - 1, 1 << 24, (1 << 31) - 1):
        F = min(62, 63 - _ceil_log2(n))
        for S in (1 << F, (1 << F) + 1, n * (1 << F) if n * (1 << F) < (1 << 63) else (1 << 63) - 1):
            for C in (0, 1, S // 2, S - 1, S):
                for U in (0, S - 1):
                    gap = _offset_estimate_gap(n, S, U, C)
                    assert 0 <= gap <= 3, (n, S, U, C, gap)
