"""Pins of the oracle's proposal step (Algorithm 2, line 4; the random-walk
proposal x_t ~ N(x_{t-1}, eps) of Sec. 5.2.3, eps read as a standard deviation).

The move is pinned against things other than itself:
  * exactness: every output coordinate is the correctly rounded value of the
    real number x + eps z (computed exactly with fractions and rounded once by
    Python's float(), an independent rounding), where z are the pinned normals
    of the particle's counter -- a step applied twice, an omitted coordinate,
    a wrong particle or iteration counter, or the normals of another purpose
    fail it;
  * scale: the sample standard deviation of the increments equals eps within
    five standard errors, for steps whose square differs from themselves, so
    a step read as a variance (eps^2) or as 2 eps fails, whatever the normals;
  * location: the increments have mean zero and do not depend on x.
"""
from fractions import Fraction

import numpy as np
import pytest

STEPS = [0.05, 0.5, 1.7]


def _exact_move(x_in, z, step):
    out = np.empty_like(x_in)
    s = Fraction(step)
    for idx in np.ndindex(x_in.shape):
        out[idx] = float(Fraction(float(x_in[idx])) + s * Fraction(float(z[idx])))
    return out


@pytest.mark.parametrize("ubits", [53, 24])
@pytest.mark.parametrize("step", STEPS)
def test_move_is_one_rounding_of_x_plus_step_z(orc, step, ubits):
    seed, t, N, D = 11, 3, 64, 5
    rng = np.random.default_rng(2)
    x = rng.normal(0.0, 3.0, size=(N, D))
    out = orc.move(x, seed, t, step, ubits=ubits)
    z = np.stack([orc.normals(seed, t, orc.ORC_MOVE, i, D, ubits) for i in range(N)])
    np.testing.assert_array_equal(out, _exact_move(x, z, step))
    # (the increments are then eps z up to one rounding of x + eps z)
    inc = (out - x) / step
    assert np.max(np.abs(inc - z)) <= 4 * np.finfo(float).eps * np.max(np.abs(out) + np.abs(x)) / step


@pytest.mark.parametrize("ubits", [53, 24])
@pytest.mark.parametrize("step", STEPS)
def test_move_increment_scale_is_step(orc, step, ubits):
    # N D = 2^16 increments from x = 0: their standard deviation is eps
    # (standard error of a normal sample's std: eps / sqrt(2 n))
    N, D = 8192, 8
    x = np.zeros((N, D))
    inc = orc.move(x, 5, 2, step, ubits=ubits).ravel()
    n = inc.size
    sd = inc.std()
    assert abs(sd - step) < 5 * step / np.sqrt(2 * n), (sd, step)
    assert abs(inc.mean()) < 5 * step / np.sqrt(n)
    # a variance reading (eps^2) or a doubled step lie far outside
    for wrong in (step * step, 2 * step):
        assert abs(sd - wrong) > 20 * step / np.sqrt(2 * n)


def test_move_increment_independent_of_position(orc):
    # the proposal is a random walk: the same counter moves every starting
    # point by the same increment, so x_t - x_{t-1} does not depend on x_{t-1}
    N, D, step = 256, 4, 0.5
    rng = np.random.default_rng(7)
    a = rng.normal(0.0, 1.0, size=(N, D))
    b = a + 1000.0 * rng.normal(0.0, 1.0, size=(N, D))
    ia = orc.move(a, 9, 4, step) - a
    ib = orc.move(b, 9, 4, step) - b
    # equal up to the roundings of x + eps z at each magnitude
    assert np.max(np.abs(ia - ib)) < 1e-9
    # and the increments differ between iterations and between seeds
    assert not np.allclose(orc.move(a, 9, 5, step) - a, ia)
    assert not np.allclose(orc.move(a, 8, 4, step) - a, ia)
    # the zero step leaves every particle where it is
    np.testing.assert_array_equal(orc.move(a, 9, 4, 0.0), a)
