"""Pins of the oracle's canonical arithmetic against mathematics (mpmath at
50 digits), not against itself.  Eq. 1 of the paper needs sin/cos of the
catalogue angles; the oracle evaluates them in degrees after an exact
reduction to [-45, 45] deg."""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle as O

mp.mp.dps = 50


def test_coefficients_are_nearest_doubles_of_taylor_terms():
    s, c = O.coefficients()
    p = mp.pi / 180
    for k in range(10):
        exact = (-1) ** k * p ** (2 * k + 1) / mp.factorial(2 * k + 1)
        assert s[k] == float(exact), k
    for k in range(11):
        exact = (-1) ** k * p ** (2 * k) / mp.factorial(2 * k)
        assert c[k] == float(exact), k


def _truth(x):
    r = mp.mpf(float(x)) * mp.pi / 180
    return mp.sin(r), mp.cos(r)


def test_sincos_deg_error_bound():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-720, 720, 3000), np.arange(-720, 721, 15.0),
                        rng.uniform(-1e-6, 1e-6, 200), 45.0 + rng.uniform(-1e-9, 1e-9, 100),
                        [0.0, -0.0, 1e-300, 89.99999999999999, 90.00000000000001]])
    s, c = O.sincos_deg(x)
    worst = 0.0
    for xi, si, ci in zip(x, s, c):
        ts, tc = _truth(xi)
        worst = max(worst, float(abs(si - ts)), float(abs(ci - tc)))
    # a degree-19/20 Horner evaluation with |t| <= 45 deg stays within 2 ulp of 1
    assert worst <= 2.3e-16


def test_sincos_deg_exact_values():
    s, c = O.sincos_deg(np.array([0.0, 90.0, 180.0, 270.0, -90.0, 360.0, 720.0]))
    np.testing.assert_array_equal(s, [0.0, 1.0, 0.0, -1.0, -1.0, 0.0, 0.0])
    np.testing.assert_array_equal(np.abs(c), [1.0, 0.0, 1.0, 0.0, 0.0, 1.0, 1.0])
    s, c = O.sincos_deg(np.array([30.0, 60.0, 45.0]))
    assert abs(s[0] - 0.5) <= 2 ** -53
    assert abs(c[1] - 0.5) <= 2 ** -53
    assert abs(s[2] - math.sqrt(0.5)) <= 2 ** -52


def test_sin_small_angle_is_relatively_accurate():
    # tiny half-radii (the threshold of Eq. 1) need relative, not absolute accuracy
    for x in [1e-12, 1.0 / 7200, 2.5 / 7200, 5.0 / 7200, 1e-3]:
        s, _ = O.sincos_deg(np.array([x]))
        ts, _ = _truth(x)
        assert abs(s[0] - float(ts)) <= 2 * abs(float(ts)) * 2 ** -52


def test_norm_ra():
    out = O.norm_ra(np.array([-10.0, 0.0, 360.0, 725.5, -1e-20, 359.5, -720.0]))
    assert out[0] == 350.0 and out[1] == 0.0 and out[2] == 0.0 and out[3] == 5.5
    assert 0.0 <= out[4] < 360.0 and out[5] == 359.5 and out[6] == 0.0


def test_unit_vectors_have_unit_norm_and_known_directions():
    rng = np.random.default_rng(3)
    ra = rng.uniform(0, 360, 5000)
    dec = rng.uniform(-90, 90, 5000)
    v = O.unitvec(ra, dec)
    assert np.max(np.abs(np.einsum("ij,ij->i", v, v) - 1.0)) < 1e-15
    v = O.unitvec(np.array([0.0, 90.0, 123.0, 0.0]), np.array([0.0, 0.0, 90.0, -90.0]))
    np.testing.assert_array_equal(v[0], [1.0, 0.0, 0.0])
    np.testing.assert_allclose(v[1], [0.0, 1.0, 0.0], atol=0)
    assert v[2][0] == 0.0 and v[2][1] == 0.0 and v[2][2] == 1.0
    assert v[3][2] == -1.0


@pytest.mark.parametrize("r", [0.1, 1.0, 1.5, 5.0, 3600.0, 648000.0])
def test_threshold_is_4_sin2_half_r(r):
    truth = 4 * mp.sin(mp.mpf(r) / 3600 * mp.pi / 180 / 2) ** 2
    got = O.threshold(r)
    assert abs(got - float(truth)) <= 4 * float(truth) * 2 ** -52
