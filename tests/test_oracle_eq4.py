"""Pins of the oracle's per-source error radii (Eq. 4, Sec. 2.1): a pair
(A_i, B_j) matches when its distance is at most 3 sqrt(e_i^2 + e_j^2).

- closed forms: pairs on one meridian (distance = |dDec|) and on the equator
  (distance = |dRA|) placed 1e-9 relative inside and outside radii built
  from Pythagorean triples that binary64 holds exactly; each misreading of
  the rule (the factor 3 dropped, errors added instead of in quadrature, the
  larger error only, one catalogue's error only) decides one of them wrongly;
- special case: constant errors reduce to the single-radius matcher;
- brute force: the cell-indexed matcher equals the all-pairs one on clumpy
  inputs around poles, the RA wrap and face vertices;
- invariants: independence of the HEALPix order, and swapping the
  catalogues transposes the set;
- the completeness condition (largest pair radius <= theta_L/8) and invalid
  errors are rejected.
"""
import math

import numpy as np
import pytest

import oracle as O


def _pairs(res):
    return set(zip(res["ia"].tolist(), res["ib"].tolist()))


# (e_a, e_b, exact 3 sqrt(e_a^2 + e_b^2)) with every value exact in binary64
TRIPLES = [(0.375, 0.5, 1.875), (0.25, 0.0, 0.75), (0.0, 0.0, 0.0), (0.625, 1.5, 4.875),
           (0.09375, 0.125, 0.46875)]


def test_pair_radius_of_exact_triples():
    for ea, eb, r in TRIPLES:
        assert O.pair_radius(ea, eb)[0] == r
    # symmetric in the two errors
    rng = np.random.default_rng(3)
    e1, e2 = rng.uniform(0, 2, 1000), rng.uniform(0, 2, 1000)
    np.testing.assert_array_equal(O.pair_radius(e1, e2), O.pair_radius(e2, e1))
    np.testing.assert_allclose(O.pair_radius(e1, e2), 3 * np.hypot(e1, e2), rtol=1e-15)


def _meridian_cases():
    """A sources on the meridian RA 37, B sources straight north of them at
    distance r (1 +- 1e-9), r from the exact triples; also on the equator."""
    ra_a, dec_a, ea, ra_b, dec_b, eb, want = [], [], [], [], [], [], []
    for k, (e1, e2, r) in enumerate(TRIPLES):
        if r == 0.0:
            continue
        for sgn in (-1.0, 1.0):
            d = r * (1.0 + sgn * 1e-9) / 3600.0
            dec0 = -40.0 + 7.0 * k + (0.5 if sgn > 0 else 0.0)
            ra_a.append(37.0); dec_a.append(dec0); ea.append(e1)
            ra_b.append(37.0); dec_b.append(dec0 + d); eb.append(e2)
            want.append(sgn < 0)
            # on the equator the distance is the RA difference
            ra0 = 100.0 + 9.0 * k + (0.5 if sgn > 0 else 0.0)
            ra_a.append(ra0); dec_a.append(0.0); ea.append(e1)
            ra_b.append(ra0 + d); dec_b.append(0.0); eb.append(e2)
            want.append(sgn < 0)
    return (np.array(ra_a), np.array(dec_a), np.array(ea), np.array(ra_b), np.array(dec_b),
            np.array(eb), np.array(want))


def test_placed_pairs_decided_by_closed_form():
    ra_a, dec_a, ea, ra_b, dec_b, eb, want = _meridian_cases()
    n = ra_a.size
    ida = np.arange(n, dtype=np.uint64) + (1 << 40)
    idb = np.arange(n, dtype=np.uint64) + (1 << 41)
    got = O.match_eq4(ra_a, dec_a, ida, ea, ra_b, dec_b, idb, eb, 8)
    got_pairs = _pairs(got)
    # the partner of A_i is B_i; sources are far apart otherwise
    for i in range(n):
        assert ((i, i) in got_pairs) == want[i], i
    assert all(a == b for a, b in got_pairs)
    # separations: the placed distance
    d = np.where(dec_a == 0.0, ra_b - ra_a, dec_b - dec_a) * 3600.0
    np.testing.assert_allclose(got["sep"], d[got["ia"]], rtol=0, atol=1e-9)


@pytest.mark.parametrize("rule", ["no_factor_3", "sum_not_quadrature", "larger_only",
                                  "a_only"])
def test_each_misreading_decides_a_placed_pair_wrongly(rule):
    """The placed pairs separate the rule from its plausible misreadings."""
    ra_a, dec_a, ea, ra_b, dec_b, eb, want = _meridian_cases()
    wrong = {"no_factor_3": np.hypot(ea, eb), "sum_not_quadrature": 3 * (ea + eb),
             "larger_only": 3 * np.maximum(ea, eb), "a_only": 3 * ea}[rule]
    d = np.where(dec_a == 0.0, ra_b - ra_a, dec_b - dec_a) * 3600.0
    assert np.any((d <= wrong) != want)


def test_constant_errors_reduce_to_one_radius():
    from paper_2301_07331_b300 import synth
    A, B = synth.patch_pair(na=8000, nb=8000, seed=11)
    ra_a, dec_a, ida = A.numpy()
    ra_b, dec_b, idb = B.numpy()
    e1, e2 = 0.2, 0.25
    r = O.pair_radius(e1, e2)[0]
    got = O.match_eq4(ra_a, dec_a, ida, np.full(ra_a.size, e1), ra_b, dec_b, idb,
                      np.full(ra_b.size, e2), 13)
    ref = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, 13, O.COMPLETE)
    assert ref["id_a"].size > 1000
    for k in ("ia", "ib", "chord2"):
        np.testing.assert_array_equal(got[k], ref[k])


def _clumpy(rng, n, spread_arcsec, centres):
    ci = rng.integers(0, len(centres), n)
    ra0 = np.array([c[0] for c in centres])[ci]
    dec0 = np.array([c[1] for c in centres])[ci]
    pa = rng.uniform(0, 2 * math.pi, n)
    dist = np.radians(spread_arcsec / 3600.0) * np.sqrt(rng.uniform(0, 1, n))
    d0 = np.radians(dec0)
    d1 = np.arcsin(np.clip(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa),
                           -1, 1))
    a1 = np.radians(ra0) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                      np.cos(dist) - np.sin(d0) * np.sin(d1))
    return np.mod(np.degrees(a1), 360.0), np.clip(np.degrees(d1), -90, 90)


@pytest.mark.parametrize("L,seed", [(4, 0), (7, 1), (10, 2), (12, 3)])
def test_complete_eq4_equals_brute_force(L, seed):
    rng = np.random.default_rng(seed)
    rmax = O.complete_max_radius(L) * 0.999
    emax = rmax / (3 * math.sqrt(2))
    pix = rng.integers(0, 12 * 4 ** L, 50).astype(np.uint64)
    ra, dec = O.pix2ang(pix, L)
    vz = math.degrees(math.asin(2.0 / 3.0))
    cen = list(zip(ra.tolist(), dec.tolist())) + [(0.0, 90.0), (45.0, -90.0), (359.9999, 10.0),
                                                  (0.0, vz), (90.0, -vz), (45.0, 0.0)]
    ra_a, dec_a = _clumpy(rng, 1500, 3 * rmax, cen)
    ra_b, dec_b = _clumpy(rng, 1500, 3 * rmax, cen)
    ea = emax * rng.uniform(0, 1, 1500) ** 2
    eb = emax * rng.uniform(0, 1, 1500)
    eb[:20] = emax  # the largest radius present
    ida = rng.integers(0, 2 ** 63, 1500).astype(np.uint64)
    idb = rng.integers(0, 2 ** 63, 1500).astype(np.uint64)
    got = O.match_eq4(ra_a, dec_a, ida, ea, ra_b, dec_b, idb, eb, L)
    ref = O.match_brute_eq4(ra_a, dec_a, ida, ea, ra_b, dec_b, idb, eb)
    assert got["id_a"].size > 300
    for k in ("ia", "ib", "chord2"):
        np.testing.assert_array_equal(got[k], ref[k])
    # radii are per source: some pairs match only thanks to their own errors
    r_fixed = O.pair_radius(np.median(ea), np.median(eb))[0]
    fixed = O.match_brute(ra_a, dec_a, ida, ra_b, dec_b, idb, r_fixed)
    assert _pairs(fixed) != _pairs(got)


def test_eq4_independent_of_order_and_transposes():
    from paper_2301_07331_b300 import synth
    A, B = synth.patch_pair(na=12000, nb=12000, seed=5)
    ra_a, dec_a, ida = A.numpy()
    ra_b, dec_b, idb = B.numpy()
    rng = np.random.default_rng(8)
    ea = rng.uniform(0.05, 0.4, ra_a.size)
    eb = rng.uniform(0.05, 0.4, ra_b.size)
    ref = None
    for L in range(3, 14):
        if O.pair_radius(ea.max(), eb.max())[0] > O.complete_max_radius(L):
            continue
        got = O.match_eq4(ra_a, dec_a, ida, ea, ra_b, dec_b, idb, eb, L)
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got["ia"], ref["ia"])
            np.testing.assert_array_equal(got["ib"], ref["ib"])
    assert ref["ia"].size > 1000
    sw = O.match_eq4(ra_b, dec_b, idb, eb, ra_a, dec_a, ida, ea, 12)
    assert _pairs(sw) == {(b, a) for a, b in _pairs(ref)}


def test_rejects_invalid_errors_and_too_large_radii():
    ra, dec, ids = np.array([10.0]), np.array([5.0]), np.array([1], np.uint64)
    ok = O.match_eq4(ra, dec, ids, [0.1], ra, dec, ids, [0.1], 12)
    assert ok["id_a"].size == 1  # a source matches its own copy
    for bad in ([-0.1], [np.nan], [np.inf]):
        with pytest.raises(O.OracleError):
            O.match_eq4(ra, dec, ids, bad, ra, dec, ids, [0.1], 12)
    emax = O.complete_max_radius(12) / 3.0
    with pytest.raises(O.OracleError):
        O.match_eq4(ra, dec, ids, [emax], ra, dec, ids, [0.01], 12)
    # zero errors: only coincident positions match
    z = O.match_eq4(np.array([10.0, 10.0]), np.array([5.0, 5.0 + 1e-12]), np.array([1, 2], np.uint64),
                    [0.0, 0.0], ra, dec, ids, [0.0], 12)
    assert _pairs(z) == {(0, 0)}
