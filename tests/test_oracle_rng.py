"""Pins of the oracle's random numbers against sources other than itself.

Philox4x32-10 is checked against cuRAND's host-side PHILOX4_32_10 generator, an
independent implementation of the same published generator (Salmon et al.,
SC'11): with the default ordering, its 32-bit output stream is the blocks
philox((0, 0, b, 0), (seed low, seed high)) for b = 0, 1, 2, ...  The library is
run, not inspected.  The Box-Muller normals are checked by distribution (KS
test, moments, independence across counters) rather than by retyping their
formula.
"""
import ctypes
import os

import numpy as np
import pytest

M32 = (1 << 32) - 1


def _curand():
    for path in (os.environ.get("CUDA_HOME", "/usr/local/cuda") + "/lib64/libcurand.so", "libcurand.so",
                 "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    pytest.skip("cuRAND host library not available")


def curand_philox_stream(seed: int, nwords: int) -> np.ndarray:
    L = _curand()
    g = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        L.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x1234567890ABCDEF, (1 << 64) - 1, 0xFFFFFFFF, 1 << 32, 977])
def test_philox_matches_curand(orc, seed):
    nblocks = 300
    ref = curand_philox_stream(seed, 4 * nblocks).reshape(nblocks, 4)
    key = [seed & M32, seed >> 32]
    for b in list(range(40)) + [99, 255, 299]:
        np.testing.assert_array_equal(orc.philox4x32_10([0, 0, b, 0], key), ref[b])


def test_philox_counter_words_all_enter(orc):
    # the pin above drives counter word 2 only; each other word must change
    # the output too (a word dropped from the round function would not)
    base = orc.philox4x32_10([5, 6, 7, 8], [9, 10])
    for j in range(4):
        c = [5, 6, 7, 8]
        c[j] ^= 1
        assert not np.array_equal(orc.philox4x32_10(c, [9, 10]), base)
    for j in range(2):
        k = [9, 10]
        k[j] ^= 1
        assert not np.array_equal(orc.philox4x32_10([5, 6, 7, 8], k), base)


def test_philox_stream_layout(orc):
    # word w of particle i, iteration t, purpose p is output w % 4 of the block
    # with counter (i, t, p << 24 | w // 4, 0) and key (seed low, seed high);
    # FP32 path: uniforms are the top 24 bits of consecutive 32-bit words,
    # FP64 path: the top 53 bits of (word 2k << 32 | word 2k + 1)
    seed, t, i = 0xDEADBEEF12345678, 7, 1234
    key = [seed & M32, seed >> 32]
    blk = orc.philox4x32_10([i, t, (orc.ORC_MOVE << 24) | 0, 0], key).astype(np.uint64)
    z = orc.normals(seed, t, orc.ORC_MOVE, i, 2, 24)
    a, b = (blk[0] >> 8) * 2.0 ** -24, (blk[1] >> 8) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log1p(-a))
    assert abs(z[0] - r * np.cos(2 * np.pi * b)) < 1e-12
    assert abs(z[1] - r * np.sin(2 * np.pi * b)) < 1e-12
    z = orc.normals(seed, t, orc.ORC_MOVE, i, 2, 53)
    a = int(((int(blk[0]) << 32) | int(blk[1])) >> 11) * 2.0 ** -53
    b = int(((int(blk[2]) << 32) | int(blk[3])) >> 11) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log1p(-a))
    assert abs(z[0] - r * np.cos(2 * np.pi * b)) < 1e-12
    assert abs(z[1] - r * np.sin(2 * np.pi * b)) < 1e-12


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
