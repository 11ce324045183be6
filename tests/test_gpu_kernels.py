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
