"""Pins of the oracle's random numbers against sources other than itself.

Philox4x64-10 is checked against numpy.random.Philox, an independent
implementation of the same published generator (Salmon et al., SC'11).  The
Box-Muller normals are checked by distribution (KS test, moments, independence
across counters) rather than by retyping their formula.
"""
import numpy as np
import pytest

M64 = (1 << 64) - 1


def numpy_block(ctr, key):
    # numpy advances the 256-bit counter before producing each 4-word block,
    # so block(c) is the first output of a generator started at c - 1.
    val = sum(int(c) << (64 * k) for k, c in enumerate(ctr))
    val = (val - 1) % (1 << 256)
    cm = [(val >> (64 * k)) & M64 for k in range(4)]
    return np.random.Philox(key=np.array([int(key[0]), int(key[1])], dtype=np.uint64),
                           counter=np.array(cm, dtype=np.uint64)).random_raw(4)


@pytest.mark.parametrize("trial", range(40))
def test_philox_matches_numpy(orc, trial):
    g = np.random.default_rng(trial)
    ctr = [int(v) for v in g.integers(0, 2**63, size=4, dtype=np.uint64)]
    key = [int(v) for v in g.integers(0, 2**63, size=2, dtype=np.uint64)]
    if trial % 4 == 1:
        ctr[0] = M64  # carry into the second word on numpy's side
    if trial % 4 == 2:
        ctr = [0, 0, 0, 0]
    if trial % 4 == 3:
        key = [M64, M64]
    np.testing.assert_array_equal(orc.philox4x64_10(ctr, key), numpy_block(ctr, key))


def test_philox_stream_layout(orc):
    # word w of particle i, iteration t, purpose p is output w%4 of the block
    # with counter (i, t, p << 32 | w // 4, 0) and key (seed, 0)
    out = orc.philox4x64_10([7, 3, (2 << 32) | 1, 0], [11, 0])
    np.testing.assert_array_equal(out, numpy_block([7, 3, (2 << 32) | 1, 0], [11, 0]))


@pytest.mark.parametrize("ubits", [53, 24])
def test_normals_distribution(orc, ubits):
    st = pytest.importorskip("scipy.stats")
    D = 8
    z = np.stack([orc.normals(5, 1, orc.ORC_MOVE, i, D, ubits) for i in range(4000)])
    flat = z.ravel()
    assert abs(flat.mean()) < 5 / np.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 5 * np.sqrt(2.0 / flat.size)
    assert st.kstest(flat, "norm").pvalue > 1e-4
    # coordinates of one particle are uncorrelated (pairs come from one
    # Box-Muller draw: cos and sin parts must still be uncorrelated)
    c = np.corrcoef(z.T)
    off = c[~np.eye(D, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(z.shape[0])


def test_normals_independent_across_counters(orc):
    a = np.array([orc.normals(1, 1, orc.ORC_MOVE, i, 4) for i in range(3000)]).ravel()
    b = np.array([orc.normals(1, 2, orc.ORC_MOVE, i, 4) for i in range(3000)]).ravel()
    c = np.array([orc.normals(1, 1, orc.ORC_INIT, i, 4) for i in range(3000)]).ravel()
    d = np.array([orc.normals(2, 1, orc.ORC_MOVE, i, 4) for i in range(3000)]).ravel()
    for other in (b, c, d):
        assert abs(np.corrcoef(a, other)[0, 1]) < 5 / np.sqrt(a.size)
    # the same counter gives the same numbers
    np.testing.assert_array_equal(orc.normals(1, 1, orc.ORC_MOVE, 17, 4), orc.normals(1, 1, orc.ORC_MOVE, 17, 4))


def test_normals_odd_dimension_prefix(orc):
    # an odd D uses the cosine half of the last pair: D=3 is a prefix of D=4
    z3 = orc.normals(9, 4, orc.ORC_MOVE, 2, 3)
    z4 = orc.normals(9, 4, orc.ORC_MOVE, 2, 4)
    np.testing.assert_array_equal(z3, z4[:3])


def test_resample_u_range(orc):
    for S in (1, 2, 3, 1000, 2**39, 2**63):
        for t in range(20):
            U = orc.resample_u(3, t, S)
            assert 0 <= U < S
    # U / S is uniform over iterations
    st = pytest.importorskip("scipy.stats")
    S = 2**40 + 12345
    us = np.array([orc.resample_u(0, t, S) / S for t in range(2000)])
    assert st.kstest(us, "uniform").pvalue > 1e-4
