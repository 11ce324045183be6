"""Pins of the oracle's matchers: the complete 8-neighbour matcher equals the
all-pairs definition of Eq. 1 (brute force) on small inputs placed to cross
many cell edges (poles, RA wrap, face vertices); it does not depend on the
HEALPix order; the quad-direction set (Algorithm 1) equals its own all-pairs
definition, is a subset of the complete set, reports each pair once and loses
no more than the plain same-cell join (Table 4's qualitative finding)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_07331_b300 import synth


def _pairs(res):
    return set(zip(res["ia"].tolist(), res["ib"].tolist()))


def _clumpy(rng, n, r_arcsec, centres):
    """Points in small clumps of a few r around given centres, so that many
    pairs straddle cell edges."""
    ci = rng.integers(0, len(centres), n)
    ra0 = np.array([c[0] for c in centres])[ci]
    dec0 = np.array([c[1] for c in centres])[ci]
    pa = rng.uniform(0, 2 * math.pi, n)
    dist = np.radians(r_arcsec / 3600.0) * 4 * np.sqrt(rng.uniform(0, 1, n))
    d0 = np.radians(dec0)
    d1 = np.arcsin(np.clip(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa), -1, 1))
    a1 = np.radians(ra0) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                      np.cos(dist) - np.sin(d0) * np.sin(d1))
    return np.mod(np.degrees(a1), 360.0), np.clip(np.degrees(d1), -90, 90)


def _centres(rng, L, k=60):
    """Pixel corners and edges at order L, poles, the RA wrap and the
    three-face vertices."""
    pix = rng.integers(0, 12 * 4 ** L, k).astype(np.uint64)
    ra, dec = O.pix2ang(pix, L)
    vz = math.degrees(math.asin(2.0 / 3.0))
    extra = [(0.0, 90.0), (45.0, -90.0), (0.0, 0.0), (359.9999, 10.0), (0.0, vz),
             (90.0, -vz), (180.0, vz), (270.0, -vz), (45.0, 0.0), (315.0, 0.0)]
    return list(zip(ra.tolist(), dec.tolist())) + extra


@pytest.mark.parametrize("L,seed", [(3, 0), (4, 1), (6, 2), (8, 3), (10, 4), (12, 5)])
def test_complete_equals_brute_force(L, seed):
    rng = np.random.default_rng(seed)
    r = O.complete_max_radius(L) * 0.999
    cen = _centres(rng, L)
    ra_a, dec_a = _clumpy(rng, 1500, r, cen)
    ra_b, dec_b = _clumpy(rng, 1500, r, cen)
    ida = rng.integers(0, 2 ** 63, 1500).astype(np.uint64)
    idb = rng.integers(0, 2 ** 63, 1500).astype(np.uint64)
    got = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, L, O.COMPLETE)
    ref = O.match_brute(ra_a, dec_a, ida, ra_b, dec_b, idb, r)
    assert got["id_a"].size > 500
    np.testing.assert_array_equal(got["ia"], ref["ia"])
    np.testing.assert_array_equal(got["ib"], ref["ib"])
    np.testing.assert_array_equal(got["chord2"], ref["chord2"])
    # output order: ascending (id_a, id_b) as unsigned
    key = got["id_a"].astype(object) * 2 ** 64 + got["id_b"].astype(object)
    assert all(key[i] <= key[i + 1] for i in range(len(key) - 1))


def test_complete_is_independent_of_order():
    A, B = synth.patch_pair(na=20000, nb=20000)
    ra_a, dec_a, ida = A.numpy()
    ra_b, dec_b, idb = B.numpy()
    r = 1.5
    ref = None
    for L in range(3, 15):
        if r > O.complete_max_radius(L):
            continue
        got = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, L, O.COMPLETE)
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got["ia"], ref["ia"])
            np.testing.assert_array_equal(got["ib"], ref["ib"])
    assert ref["id_a"].size > 10000


def test_self_match_keeps_self_pairs():
    A, _ = synth.patch_pair(na=3000, nb=10)
    ra, dec, ida = A.numpy()
    got = O.match(ra, dec, ida, ra, dec, ida, 1.0, 13, O.COMPLETE)
    assert set(range(3000)) <= set((i for i, j in _pairs(got) if i == j))


def test_empty_catalogues():
    e = np.empty(0)
    got = O.match(e, e, np.empty(0, np.uint64), np.array([1.0]), np.array([1.0]),
                  np.array([5], np.uint64), 1.0, 10, O.COMPLETE)
    assert got["id_a"].size == 0


def test_invalid_inputs_rejected():
    one = np.array([1.0])
    ids = np.array([1], np.uint64)
    with pytest.raises(O.OracleError):
        O.match(one, np.array([91.0]), ids, one, one, ids, 1.0, 10)
    with pytest.raises(O.OracleError):
        O.match(np.array([np.nan]), one, ids, one, one, ids, 1.0, 10)
    with pytest.raises(O.OracleError):
        O.match(one, one, ids, one, one, ids, -1.0, 10)
    with pytest.raises(O.OracleError):  # radius too large for complete mode
        O.match(one, one, ids, one, one, ids, 10.0, 14)


def _quad_brute(ra_a, dec_a, ra_b, dec_b, r, L, cosdec=False):
    """All-pairs statement of the quad-direction set: a pair is reported when
    the two cell sets intersect and Eq. 1 holds."""
    ca, na = O.quad_cells(ra_a, dec_a, r, L, cosdec)
    cb, nb = O.quad_cells(ra_b, dec_b, r, L, cosdec)
    ref = O.match_brute(ra_a, dec_a, np.arange(ra_a.size, dtype=np.uint64),
                        ra_b, dec_b, np.arange(ra_b.size, dtype=np.uint64), r)
    out = set()
    for i, j in zip(ref["ia"].tolist(), ref["ib"].tolist()):
        if set(ca[i, :na[i]].tolist()) & set(cb[j, :nb[j]].tolist()):
            out.add((i, j))
    return out, _pairs(ref)


@pytest.mark.parametrize("mode", [O.QUAD, O.QUAD_COS], ids=["literal", "cosdec"])
@pytest.mark.parametrize("L,seed", [(6, 0), (9, 1), (12, 2)])
def test_quad_equals_its_all_pairs_definition(L, seed, mode):
    rng = np.random.default_rng(seed)
    r = O.complete_max_radius(L) * 2.5  # quad mode has no radius limit
    cen = _centres(rng, L)
    ra_a, dec_a = _clumpy(rng, 1200, r, cen)
    ra_b, dec_b = _clumpy(rng, 1200, r, cen)
    ids = np.arange(1200, dtype=np.uint64)
    got = O.match(ra_a, dec_a, ids, ra_b, dec_b, ids, r, L, mode)
    want, full = _quad_brute(ra_a, dec_a, ra_b, dec_b, r, L, mode == O.QUAD_COS)
    gp = list(zip(got["ia"].tolist(), got["ib"].tolist()))
    assert len(gp) == len(set(gp))  # each pair once
    assert set(gp) == want
    assert want <= full


def test_quad_loses_no_more_than_same_cell_join():
    A, B = synth.fullsky_pair(na=300_000, nb=300_000)
    ra_a, dec_a, ida = A.numpy()
    ra_b, dec_b, idb = B.numpy()
    L, r = 12, 1.5
    comp = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, L, O.COMPLETE)
    quad = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, L, O.QUAD)
    pa = O.ang2pix(ra_a, dec_a, L)[comp["ia"]]
    pb = O.ang2pix(ra_b, dec_b, L)[comp["ib"]]
    same_cell = int((pa == pb).sum())
    assert _pairs(quad) <= _pairs(comp)
    assert same_cell <= quad["id_a"].size <= comp["id_a"].size
    assert comp["id_a"].size - quad["id_a"].size < 0.01 * comp["id_a"].size
    qcos = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, r, L, O.QUAD_COS)
    assert _pairs(qcos) <= _pairs(comp)
    assert same_cell <= qcos["id_a"].size


def test_jittered_recovery_rate_c1():
    """Statistical sanity: 70% of B are A offset by a 2D Gaussian of 0.3";
    the fraction recovered within 1" is 1 - exp(-r^2 / 2 sigma^2)."""
    A, B = synth.patch_pair()
    ra_a, dec_a, ida = A.numpy()
    ra_b, dec_b, idb = B.numpy()
    got = O.match(ra_a, dec_a, ida, ra_b, dec_b, idb, 1.0, 13, O.COMPLETE)
    nj = 14000
    rec = np.sum((got["ib"] < nj) & (got["ia"] == got["ib"]))
    p = 1 - math.exp(-1.0 / (2 * 0.3 ** 2))
    assert abs(rec - nj * p) < 5 * math.sqrt(nj * p * (1 - p)) + 1
