"""GPU parity of the single-step entry points against the CPU oracle (or, for
the sort and the cell table, against their plain definitions): canonical unit
vectors and nested pixels bit for bit, neighbours, quad-direction cells, the
radix sort and the run-length cell table."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2301_07331_b300 as hlc

pytestmark = pytest.mark.gpu


def _points(n, seed):
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    # edge values: poles, RA wrap, zone boundary |z| = 2/3, face corners
    vz = math.degrees(math.asin(2.0 / 3.0))
    edge_ra = np.array([0.0, 359.99999999999994, 90.0, 45.0, 180.0, 270.0, 315.0, 0.0, 135.0])
    edge_dec = np.array([90.0, -90.0, vz, -vz, 0.0, np.nextafter(vz, 0), np.nextafter(vz, 90),
                         -0.0, 89.99999999])
    k = edge_ra.size
    ra[:k], dec[:k] = edge_ra, edge_dec
    ra[k:2 * k] = rng.uniform(-720, 720, k)  # unnormalised RA
    return ra, dec


def _cuda(*arrs):
    return [torch.as_tensor(a).cuda() for a in arrs]


def test_unitvec_bit_exact():
    ra, dec = _points(300_000, 1)
    r, d = _cuda(ra, dec)
    got = hlc.hlc_unitvec(r, d).cpu().numpy()
    want = O.unitvec(ra, dec)
    np.testing.assert_array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("order", [0, 1, 5, 9, 12, 13, 14])
def test_ang2pix_bit_exact(order):
    ra, dec = _points(400_000, 10 + order)
    # add pixel centres and points a hair away from pixel edges at this order
    pix = np.random.default_rng(order).integers(0, 12 * 4 ** order, 20000).astype(np.uint64)
    pr, pd = O.pix2ang(pix, order)
    ra = np.concatenate([ra, pr, pr + 1e-12, np.clip(pd * 0 + pr - 1e-12, 0, None)])
    dec = np.concatenate([dec, pd, pd, pd])
    r, d = _cuda(ra, dec)
    for prec in (hlc.HLC_FP64, hlc.HLC_FP32_GUARD):
        got = hlc.hlc_ang2pix(r, d, order, prec).cpu().numpy().view(np.uint32)
        want = O.ang2pix(ra, dec, order)
        np.testing.assert_array_equal(got.astype(np.uint64), want)


# distances (in units of the floor's argument) at which points are placed
# from pixel edges: beyond the FP32 estimate's guard margin, inside it but
# beyond the float-float tier's, and inside both (binary64 decides)
EDGE_DELTAS = [s * d for d in (1e-2, 1e-4, 1e-6, 3e-7, 1e-7, 1e-8, 1e-10, 1e-12, 1e-13)
               for s in (1.0, -1.0)]


def _edge_points(order, n, seed):
    """Points a given distance from the decision thresholds of the nested
    ang2pix: the two equatorial diagonals ns (1/2 + ra/90) -/+ 3/4 ns z, the
    polar coordinates tp tmp and (1 - tp) tmp, RA multiples of 90 in the caps
    and the zone boundary |z| = 2/3 (Gorski et al. 2005, written out here
    from the definition, not from the library)."""
    rng = np.random.default_rng(seed)
    ns = 2.0 ** order
    ras, decs = [], []
    for dl in EDGE_DELTAS:
        # equatorial: ns (0.5 + ra/90) - s 0.75 ns z = k + dl
        z = rng.uniform(-0.66, 0.66, n)
        sgn = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
        ra0 = rng.uniform(0.0, 360.0, n)
        k = np.round(ns * (0.5 + ra0 / 90.0) - sgn * 0.75 * ns * z)
        ra = 90.0 * ((k + dl) / ns + sgn * 0.75 * z - 0.5)
        ok = (ra >= 0.0) & (ra < 360.0)
        ras.append(ra[ok]); decs.append(np.degrees(np.arcsin(z[ok])))
        # polar: tp tmp = k + dl or (1 - tp) tmp = k + dl, tmp = ns sqrt(6) sin((90-|dec|)/2)
        dec = rng.uniform(42.0, 89.999, n) * np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
        tmp = ns * math.sqrt(6.0) * np.sin(np.radians(0.5 * (90.0 - np.abs(dec))))
        kk = np.floor(rng.uniform(0.0, 1.0, n) * tmp)
        tp = (kk + dl) / tmp
        tp = np.where(rng.uniform(size=n) < 0.5, tp, 1.0 - tp)
        ntt = rng.integers(0, 4, n)
        ra = 90.0 * (ntt + tp)
        ok = (tp > 0.0) & (tp < 1.0) & (ra >= 0.0) & (ra < 360.0)
        ras.append(ra[ok]); decs.append(dec[ok])
        # polar caps at RA multiples of 90; the zone boundary
        m = 64
        ras.append(np.clip(90.0 * rng.integers(0, 4, m) + dl * 90.0, 0.0, np.nextafter(360.0, 0)))
        decs.append(rng.uniform(42.0, 89.9, m))
        zz = np.clip(2.0 / 3.0 + dl, -1.0, 1.0) * np.where(rng.uniform(size=m) < 0.5, -1.0, 1.0)
        ras.append(rng.uniform(0.0, 360.0, m)); decs.append(np.degrees(np.arcsin(zz)))
    return np.concatenate(ras), np.concatenate(decs)


@pytest.mark.parametrize("order", [0, 2, 6, 10, 12, 13, 14])
def test_ang2pix_near_pixel_edges(order):
    """Points placed 1e-2 ... 1e-13 from every kind of pixel edge: the FP32
    estimate, the float-float tier and binary64 each decide some, and every
    pixel equals the oracle's."""
    ra, dec = _edge_points(order, 2000, 100 + order)
    assert ra.size > 30000
    r, d = _cuda(ra, dec)
    want = O.ang2pix(ra, dec, order)
    for prec in (hlc.HLC_FP64, hlc.HLC_FP32_GUARD):
        got = hlc.hlc_ang2pix(r, d, order, prec).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("order", [4, 12, 14])
def test_quad_cells_of_sources_whose_copies_land_near_edges(order):
    """Sources placed so that a shifted copy (ra + R, ra - R, dec - R or
    dec + R) lands within 1e-2 ... 1e-13 of a pixel edge."""
    r = 1.5
    R = r / 3600.0
    pr, pd = _edge_points(order, 300, 200 + order)
    which = np.random.default_rng(order).integers(0, 4, pr.size)
    ra = np.where(which == 0, pr - R, np.where(which == 1, pr + R, pr))
    dec = np.where(which == 2, pd + R, np.where(which == 3, pd - R, pd))
    ok = (ra >= 0.0) & (ra < 360.0) & (np.abs(dec) <= 90.0)
    ra, dec = ra[ok], dec[ok]
    rr, dd = _cuda(ra, dec)
    want, wcnt = O.quad_cells(ra, dec, r, order, False)
    w = want.copy()
    w[w == np.uint64(2 ** 64 - 1)] = 0xFFFFFFFF
    for prec in (hlc.HLC_FP64, hlc.HLC_FP32_GUARD):
        got, cnt = hlc.hlc_quad_cells(rr, dd, r, order, prec, boundary=hlc.HLC_QUAD)
        np.testing.assert_array_equal(cnt.cpu().numpy(), wcnt)
        np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32).astype(np.uint64), w)


def test_ang2pix_rejects_bad_input():
    r, d = _cuda(np.array([1.0, 2.0]), np.array([0.0, 91.0]))
    with pytest.raises(hlc.HLCError) as e:
        hlc.hlc_ang2pix(r, d, 10)
    assert e.value.code == hlc.HLC_EINVAL
    r, d = _cuda(np.array([np.nan]), np.array([0.0]))
    with pytest.raises(hlc.HLCError):
        hlc.hlc_ang2pix(r, d, 10)


@pytest.mark.parametrize("order", [0, 1, 2, 3, 6])
def test_neighbours_all_pixels(order):
    pix = np.arange(12 * 4 ** order, dtype=np.uint64)
    got = hlc.hlc_neighbours(torch.as_tensor(pix.astype(np.int32)).cuda(), order).cpu().numpy()
    np.testing.assert_array_equal(got, O.neighbours(pix, order))


@pytest.mark.parametrize("order", [10, 12, 14])
def test_neighbours_sampled(order):
    pix = np.random.default_rng(order).integers(0, 12 * 4 ** order, 300_000).astype(np.uint64)
    # include face corners
    n = 1 << order
    corners = []
    for f in range(12):
        for x, y in [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1)]:
            corners.append(f * n * n + sum(((x >> b) & 1) << (2 * b) | ((y >> b) & 1) << (2 * b + 1)
                                           for b in range(order)))
    pix = np.concatenate([pix, np.array(corners, dtype=np.uint64)])
    got = hlc.hlc_neighbours(torch.as_tensor(pix.astype(np.uint32).view(np.int32)).cuda(),
                             order).cpu().numpy()
    np.testing.assert_array_equal(got, O.neighbours(pix, order))


@pytest.mark.parametrize("cosdec", [False, True], ids=["literal", "cosdec"])
@pytest.mark.parametrize("order,r", [(8, 30.0), (12, 1.5), (14, 1.0)])
def test_quad_cells_equal_oracle(order, r, cosdec):
    ra, dec = _points(200_000, order)
    # and sources whose shifted copies land on the RA = 0 line, the poles
    # and the zone boundary; near the poles the cos(Dec) variant's RA shift
    # grows to its 180 deg cap
    vz = math.degrees(math.asin(2.0 / 3.0))
    R = r / 3600.0
    ra = np.concatenate([ra, [R, 360.0 - R, 0.0, R * 0.5, 180.0, 45.0, 45.0],
                         np.linspace(0.0, 359.0, 40)])
    dec = np.concatenate([dec, [10.0, -10.0, 90.0 - R, -90.0 + R * 0.5, vz - R, vz + R, 0.0],
                          np.concatenate([90.0 - np.geomspace(R * 1e-3, R * 50, 20),
                                          -90.0 + np.geomspace(R * 1e-3, R * 50, 20)])])
    rr, dd = _cuda(ra, dec)
    want, wcnt = O.quad_cells(ra, dec, r, order, cosdec)
    w = want.copy()
    w[w == np.uint64(2 ** 64 - 1)] = 0xFFFFFFFF
    bnd = hlc.HLC_QUAD_COSDEC if cosdec else hlc.HLC_QUAD
    for prec in (hlc.HLC_FP64, hlc.HLC_FP32_GUARD):
        got, cnt = hlc.hlc_quad_cells(rr, dd, r, order, prec, boundary=bnd)
        np.testing.assert_array_equal(cnt.cpu().numpy(), wcnt)
        g = got.cpu().numpy().view(np.uint32).astype(np.uint64)
        np.testing.assert_array_equal(g, w)


# around the sort's tile of 4,608 keys (18 per thread x 256 threads): one
# ragged tile, exactly one full tile, a full tile plus one key, whole full
# tiles with no ragged tail, and many tiles with a ragged tail
@pytest.mark.parametrize("n", [0, 1, 2, 1000, 3840, 4607, 4608, 4609, 4608 * 3, 4608 * 7 + 5,
                               1_000_003])
@pytest.mark.parametrize("ksize,bits", [(4, 28), (4, 9), (8, 64), (8, 40)])
def test_sort_pairs_is_stable_sort(n, ksize, bits):
    rng = np.random.default_rng(n + bits)
    dt = np.uint32 if ksize == 4 else np.uint64
    hi = 2 ** bits
    keys = rng.integers(0, min(hi, 2 ** 63), n, dtype=np.uint64)
    if bits == 9:
        keys = rng.integers(0, 37, n, dtype=np.uint64) * 13  # many equal keys
    if bits == 64:
        keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) * 2 + rng.integers(0, 2, n).astype(np.uint64)
    keys = keys.astype(dt)
    vals = np.arange(n, dtype=np.uint32)
    tk = torch.as_tensor(keys.view(np.int32 if ksize == 4 else np.int64)).cuda()
    tv = torch.as_tensor(vals.view(np.int32)).cuda()
    hlc.hlc_sort_pairs(tk, tv, bits)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(tk.cpu().numpy().view(dt), keys[order])
    np.testing.assert_array_equal(tv.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("n", [0, 1, 5, 2048, 2049, 100_000])
def test_cell_table(n):
    rng = np.random.default_rng(n)
    keys = np.sort(rng.integers(0, max(1, n // 3), n).astype(np.uint32))
    uniq, start = hlc.hlc_cell_table(torch.as_tensor(keys.view(np.int32)).cuda())
    wu, wi = np.unique(keys, return_index=True)
    np.testing.assert_array_equal(uniq.cpu().numpy().view(np.uint32), wu)
    np.testing.assert_array_equal(start.cpu().numpy()[:-1], wi)
    assert int(start.cpu().numpy()[-1]) == n
