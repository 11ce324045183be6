"""Pins of the oracle's HEALPix nested scheme ("hp_nestid", Sec. 4.2, after
Gorski et al. 2005) and of its neighbour relation (the complete 8-neighbour
boundary rule), against geometry: base-face centres, the nested hierarchy,
equal area, round trips through pixel centres, symmetry, the 24 pixels with
7 neighbours, and disc containment at r = theta/8."""
import math

import numpy as np
import pytest

import oracle as O


def _uniform_sphere(rng, n):
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    return ra, dec


def test_base_face_centres():
    # north faces 0-3 at z = 2/3, phi = 45 + 90k; equatorial 4-7 at z = 0,
    # phi = 90k; south faces 8-11 at z = -2/3, phi = 45 + 90k
    dz = math.degrees(math.asin(2.0 / 3.0))
    for k in range(4):
        assert O.ang2pix([45.0 + 90 * k], [dz + 1e-6], 0)[0] == k
        assert O.ang2pix([45.0 + 90 * k], [dz - 1e-6], 0)[0] == k
        assert O.ang2pix([90.0 * k], [0.0], 0)[0] == 4 + k
        assert O.ang2pix([45.0 + 90 * k], [-dz], 0)[0] == 8 + k
    assert O.ang2pix([10.0], [90.0], 0)[0] < 4
    assert O.ang2pix([10.0], [-90.0], 0)[0] >= 8


def test_hierarchy_and_range():
    rng = np.random.default_rng(1)
    ra, dec = _uniform_sphere(rng, 200000)
    prev = O.ang2pix(ra, dec, 14)
    assert prev.max() < 12 * 4 ** 14
    for L in range(13, -1, -1):
        cur = O.ang2pix(ra, dec, L)
        np.testing.assert_array_equal(prev >> np.uint64(2), cur)
        prev = cur


def test_equal_area():
    rng = np.random.default_rng(2)
    ra, dec = _uniform_sphere(rng, 2_000_000)
    L = 3
    cnt = np.bincount(O.ang2pix(ra, dec, L).astype(np.int64), minlength=12 * 4 ** L)
    exp = ra.size / cnt.size
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    dof = cnt.size - 1
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)


@pytest.mark.parametrize("L", [0, 1, 2, 5, 8])
def test_round_trip_pixel_centres(L):
    pix = np.arange(12 * 4 ** L, dtype=np.uint64)
    ra, dec = O.pix2ang(pix, L)
    np.testing.assert_array_equal(O.ang2pix(ra, dec, L), pix)


@pytest.mark.parametrize("L", [12, 14])
def test_round_trip_sampled_high_orders(L):
    rng = np.random.default_rng(L)
    pix = rng.integers(0, 12 * 4 ** L, 100000).astype(np.uint64)
    ra, dec = O.pix2ang(pix, L)
    np.testing.assert_array_equal(O.ang2pix(ra, dec, L), pix)


@pytest.mark.parametrize("L", [1, 2, 3, 6])
def test_neighbours_symmetric_and_counted(L):
    pix = np.arange(12 * 4 ** L, dtype=np.uint64)
    nb = O.neighbours(pix, L)
    present = nb >= 0
    cnt = present.sum(1)
    assert set(np.unique(cnt)) == {7, 8}
    assert (cnt == 7).sum() == 24
    for p in range(pix.size):
        row = nb[p][present[p]]
        assert len(set(row.tolist())) == row.size and p not in row
        for q in row:
            assert p in nb[q]
    # the 7-neighbour pixels sit at the eight vertices z = +-2/3, phi = 90k
    ra, dec = O.pix2ang(pix[cnt == 7], L)
    z = np.sin(np.radians(dec))
    assert np.all(np.abs(np.abs(z) - 2.0 / 3.0) < 2.0 / 2 ** L)
    phi = np.mod(ra, 90.0)
    assert np.all(np.minimum(phi, 90.0 - phi) < 100.0 / 2 ** L)


def _offset(ra, dec, pa, dist):
    d0 = np.radians(dec)
    d1 = np.arcsin(np.clip(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa), -1, 1))
    a1 = np.radians(ra) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                     np.cos(dist) - np.sin(d0) * np.sin(d1))
    return np.mod(np.degrees(a1), 360.0), np.clip(np.degrees(d1), -90, 90)


@pytest.mark.parametrize("L", [2, 4, 7, 10, 13])
def test_disc_of_radius_theta_over_8_stays_in_neighbourhood(L):
    """The completeness condition of complete mode: any point within
    theta_L/8 of a source lies in the source's cell or one of its
    neighbours (sampled, with extra samples at the poles and face vertices)."""
    rng = np.random.default_rng(100 + L)
    n = 60000
    ra, dec = _uniform_sphere(rng, n)
    # concentrate some samples at the poles and at the three-face vertices
    k = n // 6
    dec[:k] = np.sign(rng.uniform(-1, 1, k)) * (90 - rng.uniform(0, 3.0 / 2 ** L, k) * 30)
    vz = math.degrees(math.asin(2.0 / 3.0))
    ra[k:2 * k] = 90.0 * rng.integers(0, 4, k) + rng.uniform(-1, 1, k) * 60.0 / 2 ** L
    dec[k:2 * k] = np.sign(rng.uniform(-1, 1, k)) * vz + rng.uniform(-1, 1, k) * 60.0 / 2 ** L
    ra = np.mod(ra, 360.0)
    dec = np.clip(dec, -90, 90)
    theta = math.sqrt(math.pi / 3) / 2 ** L
    dist = theta / 8 * np.sqrt(rng.uniform(0.8, 1.0, n))
    pa = rng.uniform(0, 2 * math.pi, n)
    ra2, dec2 = _offset(ra, dec, pa, dist)
    p = O.ang2pix(ra, dec, L)
    q = O.ang2pix(ra2, dec2, L)
    nb = O.neighbours(p, L)
    ok = (q == p) | np.any(nb == q.astype(np.int64)[:, None], axis=1)
    assert ok.all(), np.flatnonzero(~ok)[:5]


def test_quad_cells_follow_algorithm_1():
    """Cells of a source = distinct pixels of (ra, dec), (ra +- R, dec) and
    (ra, dec -+ R), R = r in degrees, RA wrapped, Dec clamped."""
    rng = np.random.default_rng(9)
    L, r = 10, 30.0
    ra, dec = _uniform_sphere(rng, 5000)
    ra[:10] = 360.0 - 1e-5  # RA wrap
    dec[10:20] = 90.0 - 1e-4  # north pole clamp
    cells, cnt = O.quad_cells(ra, dec, r, L)
    R = r / 3600.0
    for i in range(ra.size):
        pts = [(ra[i], dec[i]), ((ra[i] + R) % 360.0, dec[i]), ((ra[i] - R) % 360.0, dec[i]),
               (ra[i], max(dec[i] - R, -90.0)), (ra[i], min(dec[i] + R, 90.0))]
        want = sorted(set(int(O.ang2pix([a], [d], L)[0]) for a, d in pts))
        assert cells[i, :cnt[i]].tolist() == want
