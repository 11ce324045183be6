"""Pins of the oracle's match predicate (Eq. 1, d <= r, inclusive) against
closed forms and 50-digit truth, including pairs placed 1e-9 arcsec either
side of the radius, the RA wrap, the poles and antipodes."""
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

import oracle as O

mp.mp.dps = 50


def _pred(ra_a, dec_a, ra_b, dec_b, r):
    va = O.unitvec(np.array([ra_a]), np.array([dec_a]))
    vb = O.unitvec(np.array([ra_b]), np.array([dec_b]))
    c2 = O.chord2(va, vb)[0]
    return c2 <= O.threshold(r), O.sep_arcsec(c2)


def _true_sep_arcsec(ra_a, dec_a, ra_b, dec_b):
    """Eq. 1 in 50-digit arithmetic via the haversine form."""
    d2r = mp.pi / 180
    a1, d1, a2, d2 = (mp.mpf(float(x)) * d2r for x in (ra_a, dec_a, ra_b, dec_b))
    h = mp.sin((d2 - d1) / 2) ** 2 + mp.cos(d1) * mp.cos(d2) * mp.sin((a2 - a1) / 2) ** 2
    return 2 * mp.asin(mp.sqrt(h)) * 648000 / mp.pi


def test_same_meridian_is_dec_difference():
    for dec0, dd in [(0.0, 1.0 / 3600), (45.0, 0.5 / 3600), (-60.0, 2.0 / 3600), (89.9, 0.0002)]:
        ok, sep = _pred(123.0, dec0, 123.0, dec0 + dd, 10.0)
        exact = float((Fraction(dec0 + dd) - Fraction(dec0)) * 3600)
        assert ok and abs(sep - exact) < 1e-9


def test_equator_is_ra_difference():
    ok, sep = _pred(10.0, 0.0, 10.0 + 1.0 / 3600, 0.0, 1.5)
    exact = float((Fraction(10.0 + 1.0 / 3600) - Fraction(10.0)) * 3600)
    assert ok and abs(sep - exact) < 1e-9


def test_pole_matches_for_any_ra():
    ok, sep = _pred(10.0, 90.0, 200.0, 90.0, 1e-3)
    assert ok and sep == 0.0
    ok, sep = _pred(0.0, -90.0, 359.0, -90.0, 1e-3)
    assert ok and sep == 0.0


def test_ra_wrap():
    ok1, sep = _pred(359.9999, 0.0, 0.0001, 0.0, 1.0)
    assert ok1 and abs(sep - 0.72) < 1e-6
    ok2, _ = _pred(359.9999, 0.0, 0.0001, 0.0, 0.5)
    assert not ok2


def test_antipodes_do_not_false_positive():
    ok, sep = _pred(0.0, 0.0, 180.0, 0.0, 3600.0)
    assert not ok and abs(sep - 648000.0) < 1e-6
    ok, _ = _pred(0.0, 0.0, 180.0, 0.0, 648000.0)
    assert ok
    ok, _ = _pred(12.0, 30.0, 192.0, -30.0 + 1e-6, 3600.0 * 179.9)
    assert not ok


@pytest.mark.parametrize("r", [1.0, 1.5, 5.0])
def test_meridian_pairs_one_nanoarcsec_from_r(r):
    rng = np.random.default_rng(int(r * 10))
    for _ in range(300):
        ra = float(rng.uniform(0, 360))
        dec = float(rng.uniform(-89.0, 89.0))
        for sgn in (-1, 1):
            target = Fraction(dec) + Fraction(r) / 3600 + sgn * Fraction(1, 3600 * 10 ** 9)
            dec_b = float(target)
            delta = Fraction(dec_b) - Fraction(dec)
            margin = (delta - Fraction(r) / 3600) * 3600
            assert abs(margin) >= Fraction(5, 10 ** 10)
            ok, _ = _pred(ra, dec, ra, dec_b, r)
            assert ok == (margin <= 0)


def test_general_pairs_agree_with_truth_outside_tiny_band():
    rng = np.random.default_rng(11)
    r = 1.5
    disagreements = 0
    for _ in range(400):
        ra = float(rng.uniform(0, 360))
        dec = float(np.degrees(np.arcsin(rng.uniform(-1, 1))))
        pa = mp.mpf(float(rng.uniform(0, 2 * np.pi)))
        dist = (mp.mpf(r) + mp.mpf(float(rng.uniform(-2e-9, 2e-9)))) / 3600 * mp.pi / 180
        d0 = mp.mpf(dec) * mp.pi / 180
        d1 = mp.asin(mp.sin(d0) * mp.cos(dist) + mp.cos(d0) * mp.sin(dist) * mp.cos(pa))
        a1 = mp.mpf(ra) * mp.pi / 180 + mp.atan2(mp.sin(pa) * mp.sin(dist) * mp.cos(d0),
                                                 mp.cos(dist) - mp.sin(d0) * mp.sin(d1))
        ra_b = float(mp.fmod(a1 * 180 / mp.pi + 360, 360))
        dec_b = float(d1 * 180 / mp.pi)
        truth = _true_sep_arcsec(ra, dec, ra_b, dec_b)
        ok, sep = _pred(ra, dec, ra_b, dec_b, r)
        assert abs(sep - float(truth)) < 1e-8
        if ok != (truth <= r):
            disagreements += 1
            # the canonical FP64 decision may only differ within its error bound
            assert abs(truth - r) < mp.mpf("1e-9")
    assert disagreements <= 2


def test_reported_separation_accuracy():
    rng = np.random.default_rng(5)
    for _ in range(200):
        ra, dec = float(rng.uniform(0, 360)), float(rng.uniform(-89, 89))
        ra_b = (ra + float(rng.uniform(-1e-3, 1e-3))) % 360.0
        dec_b = dec + float(rng.uniform(-1e-3, 1e-3))
        _, sep = _pred(ra, dec, ra_b, dec_b, 10.0)
        assert abs(sep - float(_true_sep_arcsec(ra, dec, ra_b, dec_b))) < 1e-8
