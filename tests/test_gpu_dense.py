"""GPU parity on dense workloads (Plummer clusters): the FP32 complete form
orders dense offset-table cells by fine key and gives the dense A cells to
the tile kernel (B tiles staged in shared memory by bulk copies).  The match
set must equal the oracle's bit for bit, separations within 1e-6 arcsec; at
a larger size, where the oracle is too slow, the FP32 form must equal the
binary64 form (an independent path: fully sorted, no tiles)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2301_07331_b300 as hlc
from paper_2301_07331_b300 import synth

pytestmark = pytest.mark.gpu

SEP_TOL = 1e-6  # arcsec


def _run(A, B, r, L, prec, **kw):
    plan = hlc.hlc_plan((A.ra, A.dec, A.id), (B.ra, B.dec, B.id), r, L, precision=prec, **kw)
    try:
        res = hlc.hlc_match(plan)
    finally:
        hlc.hlc_free(plan)
    ia = res["id_a"].cpu().numpy().view(np.uint64)
    ib = res["id_b"].cpu().numpy().view(np.uint64)
    sep = None if res["sep"] is None else res["sep"].cpu().numpy()
    return ia, ib, sep, res["stats"]


@pytest.mark.parametrize("L", [12, 13])
@pytest.mark.parametrize("prec", [hlc.HLC_FP32_GUARD, hlc.HLC_FP64])
def test_clusters_equal_oracle(L, prec):
    # 3 clusters of 50k members (cores ~1.4e7 per sq deg) in a 350k sky:
    # at order 12 a core cell holds ~3000 A sources and its neighbourhood
    # ~13000 B sources (several staged rounds and A passes)
    A, B = synth.clustered_pair(seed=77, na=350_000, nb=260_000, n_clusters=3, members=50_000,
                                device="cuda")
    want = O.match(*A.numpy(), *B.numpy(), 1.0, L, O.COMPLETE)
    ia, ib, sep, st = _run(A, B, 1.0, L, prec)
    np.testing.assert_array_equal(ia, want["id_a"])
    np.testing.assert_array_equal(ib, want["id_b"])
    assert np.max(np.abs(sep - want["sep"])) <= SEP_TOL
    assert want["id_a"].size > 100_000
    if prec == hlc.HLC_FP32_GUARD:
        assert st["dense_entries_b"] > 0
        assert st["tile_items"] > 0 and st["tile_entries_a"] >= 32 * st["tile_items"]
        assert st["band_candidates"] > 0


def test_clusters_fp32_equals_fp64_at_scale():
    A, B = synth.clustered_pair(seed=78, na=6_000_000, nb=4_500_000, n_clusters=40,
                                members=50_000, device="cuda")
    a32, b32, s32, st32 = _run(A, B, 1.0, 13, hlc.HLC_FP32_GUARD)
    a64, b64, s64, st64 = _run(A, B, 1.0, 13, hlc.HLC_FP64)
    np.testing.assert_array_equal(a32, a64)
    np.testing.assert_array_equal(b32, b64)
    assert np.max(np.abs(s32 - s64)) <= SEP_TOL
    assert st32["tile_items"] > 100
    # sampled A sources: all their B matches by brute force in the oracle
    rng = np.random.default_rng(5)
    ra_a, dec_a, id_a = A.numpy()
    ra_b, dec_b, id_b = B.numpy()
    pick = rng.choice(ra_a.size, 300, replace=False)
    want = O.match(ra_a[pick], dec_a[pick], id_a[pick], ra_b, dec_b, id_b, 1.0, 13, O.COMPLETE)
    sel = np.isin(a32, id_a[pick])
    np.testing.assert_array_equal(a32[sel], want["id_a"])
    np.testing.assert_array_equal(b32[sel], want["id_b"])


def test_empty_neighbourhoods_and_single_dense_cell():
    # every A source in one dense fine cell, B empty around it, then B dense
    ra = np.full(3000, 150.0) + np.linspace(0, 1e-4, 3000)
    dec = np.full(3000, 20.0)
    ids = np.arange(3000, dtype=np.uint64) + (1 << 40)
    far = (np.full(100, 10.0), np.full(100, -40.0), np.arange(100, dtype=np.uint64))
    for B in [far, (ra[::2] + 1e-6, dec[::2], ids[::2] + 7)]:
        want = O.match(ra, dec, ids, *B, 1.0, 13, O.COMPLETE)
        A_ = tuple(torch.as_tensor(np.asarray(x).view(np.int64) if x.dtype == np.uint64 else x)
                   .cuda() for x in (ra, dec, ids))
        B_ = tuple(torch.as_tensor(np.asarray(x).view(np.int64) if x.dtype == np.uint64 else x)
                   .cuda() for x in B)
        plan = hlc.hlc_plan(A_, B_, 1.0, 13, precision=hlc.HLC_FP32_GUARD)
        try:
            res = hlc.hlc_match(plan)
        finally:
            hlc.hlc_free(plan)
        np.testing.assert_array_equal(res["id_a"].cpu().numpy().view(np.uint64), want["id_a"])
        np.testing.assert_array_equal(res["id_b"].cpu().numpy().view(np.uint64), want["id_b"])
