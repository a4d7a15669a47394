"""Pins of the oracle's Sequential Nearly Sort (Algorithm 8, Sec. 4.2).

S-NS is defined by its two-cursor loop; it is pinned by hand-worked cases
(tests/golden/sns_small.txt), by Definition 1 of the paper (the keys come out
as an ascending Nearly-Sorted sequence: every zero before every positive
count), and, over every key vector of small N, by a different statement of
the same result: the non-positive rows keep their order at the left end and
the positive rows appear in reverse order at the right end.  The N-R local
step (S-NS then S-R) gives the rows of S-R with the survivors in reverse
order."""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(s):
    return np.array([ord(r) for r in s.split(",")], dtype=np.int64)[:, None]


def _labels(x):
    return ",".join(chr(int(v)) for v in x[:, 0])


def test_nearly_sort_golden(orc):
    with open(os.path.join(GOLDEN, "sns_small.txt")) as f:
        cases = [[p.strip() for p in ln.split("|")] for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(cases) >= 5
    for nc, rows, rows_ns, nc_ns, rows_nr in cases:
        nc = np.array([int(v) for v in nc.split(",")], dtype=np.int32)
        k, x = orc.nearly_sort(nc, _rows(rows))
        assert _labels(x) == rows_ns
        assert ",".join(str(int(v)) for v in k) == nc_ns
        assert _labels(orc.redistribute(k, x)) == rows_nr


def is_ascending_nearly_sorted(k):
    """Definition 1: [0, ..., 0, g_0, ..., g_{m-1}] with every g_i > 0."""
    pos = k > 0
    m = int(pos.sum())
    return bool(np.all(k[: k.size - m] == 0) and np.all(pos[k.size - m:]))


@pytest.mark.parametrize("N", range(1, 8))
def test_nearly_sort_every_key_vector(orc, N):
    x = np.arange(N, dtype=np.int64)[:, None] * 7 + 3
    for keys in itertools.product((0, 1, 2, 3), repeat=N):
        nc = np.array(keys, dtype=np.int32)
        k, xn = orc.nearly_sort(nc, x)
        assert is_ascending_nearly_sorted(k), keys
        pos = nc > 0
        want_x = np.concatenate([x[~pos], x[pos][::-1]])
        want_k = np.concatenate([nc[~pos], nc[pos][::-1]])
        assert np.array_equal(xn, want_x), keys
        assert np.array_equal(k, want_k), keys


def test_nearly_sort_rows_any_width(orc):
    g = np.random.default_rng(4)
    for N, width in ((1000, 3), (4097, 16), (257, 1)):
        nc = g.integers(-1, 4, size=N).astype(np.int32)  # Algorithm 8 sends every non-positive key left
        x = g.standard_normal((N, width)).astype(np.float32)
        k, xn = orc.nearly_sort(nc, x)
        pos = nc > 0
        assert np.array_equal(xn, np.concatenate([x[~pos], x[pos][::-1]]))
        assert np.array_equal(np.sort(k), np.sort(nc))


@pytest.mark.parametrize("N", range(1, 7))
def test_nr_local_step_reverses_the_survivors(orc, N):
    """Over every composition of N: S-R of the S-NS output is the stable
    repeat of the survivors taken in reverse index order, and the same
    multiset of rows as S-R of the input."""
    x = (np.arange(N, dtype=np.int64) + 10)[:, None]
    for keys in itertools.product(range(N + 1), repeat=N):
        if sum(keys) != N:
            continue
        nc = np.array(keys, dtype=np.int32)
        k, xn = orc.nearly_sort(nc, x)
        got = orc.redistribute(k, xn)
        pos = np.nonzero(nc)[0][::-1]
        assert np.array_equal(got, np.repeat(x[pos], nc[pos], axis=0)), keys
        assert np.array_equal(np.sort(got[:, 0]), np.sort(orc.redistribute(nc, x)[:, 0])), keys
