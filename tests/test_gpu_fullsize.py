"""Parity at the benchmark's full size and launch configuration: full sky,
A = B = 10M sources, r = 1.5 arcsec, fine order 12, coarse order 4.  The
oracle cannot run all of it in seconds, so (1) the FP32 guard form must give
exactly the binary64 form's rows (two independent GPU paths), and (2) for
the A sources inside sampled sky boxes (equator, galactic centre, the RA
0/360 wrap, the north polar cap) the rows must equal the oracle's, run on
those A sources and every B source near the box, in both boundary modes.
The bulge recipe at order 14 gets the same two checks."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2301_07331_b300 as hlc
from paper_2301_07331_b300 import synth

pytestmark = pytest.mark.gpu

SEP_TOL = 1e-6  # arcsec
R, L, LC = 1.5, 12, 4


@pytest.fixture(scope="module")
def sky():
    A, B = synth.fullsky_pair(na=10_000_000, nb=10_000_000, device="cuda")
    return A, B


def _run(A, B, prec, mode=hlc.HLC_COMPLETE8):
    plan = hlc.hlc_plan(A, B, R, L, coarse_level=LC, boundary=mode, precision=prec)
    try:
        res = hlc.hlc_match(plan)
    finally:
        hlc.hlc_free(plan)
    return (res["id_a"].cpu().numpy().view(np.uint64), res["id_b"].cpu().numpy().view(np.uint64),
            res["sep"].cpu().numpy(), res["stats"])


@pytest.mark.parametrize("mode", [hlc.HLC_COMPLETE8, hlc.HLC_QUAD, hlc.HLC_QUAD_COSDEC])
def test_fp32_form_equals_fp64_form(sky, mode):
    A, B = sky
    a32, b32, s32, st = _run(A, B, hlc.HLC_FP32_GUARD, mode)
    a64, b64, s64, _ = _run(A, B, hlc.HLC_FP64, mode)
    np.testing.assert_array_equal(a32, a64)
    np.testing.assert_array_equal(b32, b64)
    assert np.max(np.abs(s32 - s64)) <= SEP_TOL
    # sorted by (id_a, id_b)
    key_ok = (a32[1:] > a32[:-1]) | ((a32[1:] == a32[:-1]) & (b32[1:] >= b32[:-1]))
    assert key_ok.all()
    assert st["matches"] == a32.size
    if mode == hlc.HLC_COMPLETE8:
        assert a32.size > 5_000_000


def _in_ra(ra, lo, hi):
    return (ra >= lo) & (ra < hi) if lo < hi else (ra >= lo) | (ra < hi)


BOXES = [  # (ra_lo, ra_hi, dec_lo, dec_hi); ra_lo > ra_hi wraps through 0
    (10.0, 11.0, 0.0, 1.0),
    (265.9, 266.9, -29.4, -28.4),   # the galactic centre (densest)
    (359.6, 0.4, 20.0, 20.8),
    (0.0, 360.0, 89.6, 90.0),       # north polar cap
]


@pytest.mark.parametrize("mode", [hlc.HLC_COMPLETE8, hlc.HLC_QUAD, hlc.HLC_QUAD_COSDEC])
@pytest.mark.parametrize("box", BOXES)
def test_sampled_boxes_equal_oracle(sky, box, mode):
    A, B = sky
    ia, ib, sp, _ = _run(A, B, hlc.HLC_FP32_GUARD, mode)
    ra_a, dec_a, id_a = A.numpy()
    ra_b, dec_b, id_b = B.numpy()
    lo, hi, d0, d1 = box
    sa = _in_ra(ra_a, lo, hi) & (dec_a >= d0) & (dec_a < d1)
    m = 0.01  # deg: far more than r
    cosd = max(np.cos(np.radians(max(abs(d0), abs(d1)) + m)), 1e-3)
    if hi - lo == 360.0 or d1 + m >= 90.0:
        sb = dec_b >= d0 - m
    else:
        sb = (_in_ra(ra_b, (lo - m / cosd) % 360.0, (hi + m / cosd) % 360.0)
              & (dec_b >= d0 - m) & (dec_b < d1 + m))
    assert sa.sum() > 20
    want = O.match(ra_a[sa], dec_a[sa], id_a[sa], ra_b[sb], dec_b[sb], id_b[sb], R, L,
                   mode)  # (the oracle's mode numbers are the library's)
    sel = np.isin(ia, id_a[sa])
    np.testing.assert_array_equal(ia[sel], want["id_a"])
    np.testing.assert_array_equal(ib[sel], want["id_b"])
    assert np.max(np.abs(sp[sel] - want["sep"]), initial=0.0) <= SEP_TOL


# Order 14 (32-bit keys, every key bit in use) on the dense bulge recipe:
# A = B = 8M, r = 1 arcsec, coarse order 4.
RB, LB, LCB = 1.0, 14, 4


@pytest.fixture(scope="module")
def bulge():
    return synth.bulge_pair(na=8_000_000, nb=8_000_000, device="cuda")


def _run_bulge(A, B, prec):
    plan = hlc.hlc_plan(A, B, RB, LB, coarse_level=LCB, precision=prec)
    try:
        res = hlc.hlc_match(plan)
    finally:
        hlc.hlc_free(plan)
    return (res["id_a"].cpu().numpy().view(np.uint64), res["id_b"].cpu().numpy().view(np.uint64),
            res["sep"].cpu().numpy())


def test_bulge_order14_fp32_equals_fp64_and_oracle_boxes(bulge):
    A, B = bulge
    a32, b32, s32 = _run_bulge(A, B, hlc.HLC_FP32_GUARD)
    a64, b64, s64 = _run_bulge(A, B, hlc.HLC_FP64)
    np.testing.assert_array_equal(a32, a64)
    np.testing.assert_array_equal(b32, b64)
    assert np.max(np.abs(s32 - s64)) <= SEP_TOL
    assert a32.size > 2_000_000
    ra_a, dec_a, id_a = A.numpy()
    ra_b, dec_b, id_b = B.numpy()
    # the galactic centre (densest) and a box on the disk away from it
    for lo, hi, d0, d1 in [(266.30, 266.50, -29.10, -28.90), (100.0, 100.5, 10.0, 10.5)]:
        sa = (ra_a >= lo) & (ra_a < hi) & (dec_a >= d0) & (dec_a < d1)
        m = 0.01
        sb = (ra_b >= lo - m) & (ra_b < hi + m) & (dec_b >= d0 - m) & (dec_b < d1 + m)
        assert sa.sum() > 20
        want = O.match(ra_a[sa], dec_a[sa], id_a[sa], ra_b[sb], dec_b[sb], id_b[sb], RB, LB,
                       O.COMPLETE)
        sel = np.isin(a32, id_a[sa])
        np.testing.assert_array_equal(a32[sel], want["id_a"])
        np.testing.assert_array_equal(b32[sel], want["id_b"])
        assert np.max(np.abs(s32[sel] - want["sep"]), initial=0.0) <= SEP_TOL
