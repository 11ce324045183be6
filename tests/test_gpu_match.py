"""End-to-end GPU parity of hlc_plan / hlc_match against the CPU oracle: the
sorted (id_a, id_b) rows must be identical and every separation within
1e-6 arcsec, in both boundary modes and both precisions, on the small patch
workload, a reduced full-sky workload, inputs placed on cell edges, poles
and the RA wrap, pairs placed a hair from the radius, and edge cases."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2301_07331_b300 as hlc
from paper_2301_07331_b300 import synth

pytestmark = pytest.mark.gpu

SEP_TOL = 1e-6  # arcsec


def _gpu_match(A, B, r, L, mode, prec, device_inputs=True, **kw):
    def dev(X):
        ra, dec, ids = X
        if device_inputs:
            return (torch.as_tensor(ra).cuda(), torch.as_tensor(dec).cuda(),
                    torch.as_tensor(np.asarray(ids).view(np.int64)).cuda())
        return (ra, dec, ids)
    plan = hlc.hlc_plan(dev(A), dev(B), r, L, boundary=mode, precision=prec, **kw)
    try:
        res = hlc.hlc_match(plan)
    finally:
        hlc.hlc_free(plan)
    return (res["id_a"].cpu().numpy().view(np.uint64), res["id_b"].cpu().numpy().view(np.uint64),
            None if res["sep"] is None else res["sep"].cpu().numpy(), res["stats"])


def _check(A, B, r, L, mode, prec, **kw):
    want = O.match(*A, *B, r, L, mode)
    ia, ib, sep, st = _gpu_match(A, B, r, L, mode, prec, **kw)
    np.testing.assert_array_equal(ia, want["id_a"])
    np.testing.assert_array_equal(ib, want["id_b"])
    if sep is not None and sep.size:
        assert np.max(np.abs(sep - want["sep"])) <= SEP_TOL
    return want, st


MODES = [(hlc.HLC_COMPLETE8, hlc.HLC_FP64), (hlc.HLC_COMPLETE8, hlc.HLC_FP32_GUARD),
         (hlc.HLC_QUAD, hlc.HLC_FP64), (hlc.HLC_QUAD, hlc.HLC_FP32_GUARD),
         (hlc.HLC_QUAD_COSDEC, hlc.HLC_FP64), (hlc.HLC_QUAD_COSDEC, hlc.HLC_FP32_GUARD)]
assert O.QUAD == hlc.HLC_QUAD and O.QUAD_COS == hlc.HLC_QUAD_COSDEC  # same mode numbers


@pytest.mark.parametrize("mode,prec", MODES)
def test_patch_workload(mode, prec):
    A, B = synth.patch_pair()
    want, st = _check(A.numpy(), B.numpy(), 1.0, 13, mode, prec)
    assert want["id_a"].size > 13000
    assert st["matches"] == want["id_a"].size


@pytest.mark.parametrize("mode,prec", MODES)
def test_fullsky_reduced(mode, prec):
    A, B = synth.fullsky_pair(na=400_000, nb=400_000)
    want, st = _check(A.numpy(), B.numpy(), 1.5, 12, mode, prec)
    assert want["id_a"].size > 100_000
    if prec == hlc.HLC_FP32_GUARD:
        assert st["band_candidates"] < 0.2 * want["id_a"].size


def _clumps(rng, n, r, L, k=80):
    pix = rng.integers(0, 12 * 4 ** L, k).astype(np.uint64)
    cra, cdec = O.pix2ang(pix, L)
    vz = math.degrees(math.asin(2 / 3))
    cra = np.concatenate([cra, [0.0, 45.0, 359.9999, 0.0, 90.0, 180.0, 270.0, 45.0]])
    cdec = np.concatenate([cdec, [90.0, -90.0, 10.0, vz, -vz, vz, -vz, 0.0]])
    ci = rng.integers(0, cra.size, n)
    pa = rng.uniform(0, 2 * math.pi, n)
    dist = np.radians(r / 3600) * 4 * np.sqrt(rng.uniform(0, 1, n))
    d0 = np.radians(cdec[ci])
    d1 = np.arcsin(np.clip(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa), -1, 1))
    a1 = np.radians(cra[ci]) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                          np.cos(dist) - np.sin(d0) * np.sin(d1))
    return np.mod(np.degrees(a1), 360.0), np.clip(np.degrees(d1), -90, 90)


@pytest.mark.parametrize("L", [3, 6, 10, 13])
@pytest.mark.parametrize("mode,prec", MODES)
def test_cell_edges_poles_wrap(L, mode, prec):
    rng = np.random.default_rng(L)
    r = O.complete_max_radius(L) * 0.99
    ra_a, dec_a = _clumps(rng, 3000, r, L)
    ra_b, dec_b = _clumps(rng, 3000, r, L)
    ida = rng.integers(0, 2 ** 63, 3000).astype(np.uint64) | np.uint64(2 ** 63)
    idb = rng.integers(0, 2 ** 63, 3000).astype(np.uint64)
    _check((ra_a, dec_a, ida), (ra_b, dec_b, idb), r, L, mode, prec)


@pytest.mark.parametrize("prec", [hlc.HLC_FP64, hlc.HLC_FP32_GUARD])
def test_pairs_a_hair_from_the_radius(prec):
    """B sources placed at r(1 +- 1e-9) and r(1 +- 1e-7) from A along random
    position angles: the FP32 bulk test cannot decide them, the recheck must."""
    rng = np.random.default_rng(77)
    n = 20000
    r = 1.5
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-0.999, 0.999, n)))
    fac = rng.choice([1 - 1e-9, 1 + 1e-9, 1 - 1e-7, 1 + 1e-7, 0.5, 0.999999], n)
    pa = rng.uniform(0, 2 * math.pi, n)
    dist = np.radians(r * fac / 3600)
    d0 = np.radians(dec)
    d1 = np.arcsin(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa))
    a1 = np.radians(ra) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                     np.cos(dist) - np.sin(d0) * np.sin(d1))
    ra_b, dec_b = np.mod(np.degrees(a1), 360), np.degrees(d1)
    ids = np.arange(n, dtype=np.uint64)
    want, st = _check((ra, dec, ids), (ra_b, dec_b, ids), r, 12, hlc.HLC_COMPLETE8, prec)
    assert 0.3 * n < want["id_a"].size < n


@pytest.mark.parametrize("r", [0.1, 1.5, 5.0, 15.0])
def test_guard_band_decisions_near_the_radius(r):
    """Pairs at r (1 + eps), |eps| log-uniform in [1e-8, 1e-3] (a fifth of
    them within a decade above the float-float window, 1e-6 r + 1e-7 arcsec),
    a tenth of them within 0.15 deg of a pole: the FP32 form (FP32 test,
    float-float recheck, binary64 for the undecided) must give the oracle's
    rows, and the float-float step must decide most candidates."""
    rng = np.random.default_rng(int(r * 100) + 5)
    n = 200_000
    ra = rng.uniform(0, 360, n)
    dec = np.degrees(np.arcsin(rng.uniform(-0.999, 0.999, n)))
    polar = rng.random(n) < 0.1
    dec[polar] = rng.choice([-1.0, 1.0], polar.sum()) * rng.uniform(89.85, 89.95, polar.sum())
    eps = np.exp(rng.uniform(np.log(1e-8), np.log(1e-3), n)) * rng.choice([-1.0, 1.0], n)
    pa = rng.uniform(0, 2 * math.pi, n)
    dist = np.radians(r * (1 + eps) / 3600)
    d0 = np.radians(dec)
    d1 = np.arcsin(np.sin(d0) * np.cos(dist) + np.cos(d0) * np.sin(dist) * np.cos(pa))
    a1 = np.radians(ra) + np.arctan2(np.sin(pa) * np.sin(dist) * np.cos(d0),
                                     np.cos(dist) - np.sin(d0) * np.sin(d1))
    ra_b, dec_b = np.mod(np.degrees(a1), 360), np.degrees(d1)
    ids = np.arange(n, dtype=np.uint64)
    L = 12 if r < 10 else 10
    want, st = _check((ra, dec, ids), (ra_b, dec_b, ids), r, L, hlc.HLC_COMPLETE8,
                      hlc.HLC_FP32_GUARD)
    # (half the placed pairs match; the crowded polar rings add neighbours)
    assert want["id_a"].size > 0.4 * n
    assert st["band_candidates"] > 0.5 * n
    # binary64 is left with the pairs inside the window (here counted with
    # twice its width), near a pole, or not "nearby" (RA or Dec difference
    # above 20 arcsec), and with no others
    m = 1e-6 * r + 1e-7
    dra = np.abs(np.mod(ra_b - ra + 180.0, 360.0) - 180.0)
    undecidable = ((np.abs(eps) * r <= 2 * m) | (np.abs(dec) > 89.9) | (np.abs(dec_b) > 89.9)
                   | (dra > 20 / 3600) | (np.abs(dec_b - dec) > 20 / 3600))
    # (slack: the polar rings' own neighbour pairs inside the FP32 band)
    assert st["band_fp64"] <= undecidable.sum() + 0.05 * n


@pytest.mark.parametrize("prec", [hlc.HLC_FP64, hlc.HLC_FP32_GUARD])
def test_torch_allocator_callback(prec):
    A, B = synth.patch_pair(na=8000, nb=8000)
    _check(A.numpy(), B.numpy(), 1.0, 13, hlc.HLC_COMPLETE8, prec, torch_alloc=True)


@pytest.mark.parametrize("prec", [hlc.HLC_FP64, hlc.HLC_FP32_GUARD])
def test_self_match_and_host_inputs(prec):
    A, _ = synth.patch_pair(na=5000, nb=10)
    X = A.numpy()
    want, _ = _check(X, X, 1.0, 13, hlc.HLC_COMPLETE8, prec, device_inputs=False)
    assert want["id_a"].size >= 5000


def test_empty_catalogues():
    e = (np.empty(0), np.empty(0), np.empty(0, np.uint64))
    one = (np.array([10.0]), np.array([10.0]), np.array([7], np.uint64))
    for A, B in [(e, e), (e, one), (one, e)]:
        for mode, prec in MODES:
            ia, ib, sep, st = _gpu_match(A, B, 1.0, 10, mode, prec, device_inputs=False)
            assert ia.size == 0 and st["matches"] == 0


def test_invalid_inputs():
    ok = (np.array([10.0, 20.0]), np.array([0.0, 1.0]), np.array([1, 2], np.uint64))
    bad_dec = (np.array([10.0]), np.array([90.5]), np.array([1], np.uint64))
    bad_nan = (np.array([np.inf]), np.array([0.0]), np.array([1], np.uint64))
    for B in (bad_dec, bad_nan):
        with pytest.raises(hlc.HLCError) as e:
            _gpu_match(ok, B, 1.0, 10, hlc.HLC_COMPLETE8, hlc.HLC_FP64, device_inputs=False)
        assert e.value.code == hlc.HLC_EINVAL
    with pytest.raises(hlc.HLCError) as e:  # radius above theta/8 in complete mode
        _gpu_match(ok, ok, 10.0, 14, hlc.HLC_COMPLETE8, hlc.HLC_FP64)
    assert e.value.code == hlc.HLC_EINVAL
    with pytest.raises(hlc.HLCError):
        _gpu_match(ok, ok, -1.0, 10, hlc.HLC_COMPLETE8, hlc.HLC_FP64)
    with pytest.raises(hlc.HLCError):
        _gpu_match(ok, ok, 1.0, 15, hlc.HLC_COMPLETE8, hlc.HLC_FP64)


def test_duplicate_ids_and_unsorted_ra():
    rng = np.random.default_rng(3)
    n = 4000
    ra = rng.uniform(-360, 720, n)  # RA outside [0, 360) is folded
    dec = rng.uniform(-1, 1, n)
    ids = rng.integers(0, 50, n).astype(np.uint64)  # many equal ids
    ra_b = ra + rng.normal(0, 1e-4, n)
    dec_b = dec + rng.normal(0, 1e-4, n)
    want = O.match(ra, dec, ids, ra_b, dec_b, ids, 1.0, 12, O.COMPLETE)
    ia, ib, sep, _ = _gpu_match((ra, dec, ids), (ra_b, dec_b, ids), 1.0, 12,
                                hlc.HLC_COMPLETE8, hlc.HLC_FP32_GUARD)
    np.testing.assert_array_equal(ia, want["id_a"])
    np.testing.assert_array_equal(ib, want["id_b"])
    # equal (id_a, id_b) rows may come in any order: compare sorted separations per key
    key = ia.astype(object) * 2 ** 64 + ib.astype(object)
    for k in set(key[:500]):
        m = key == k
        np.testing.assert_allclose(np.sort(sep[m]), np.sort(want["sep"][m]), atol=SEP_TOL, rtol=0)


@pytest.mark.parametrize("prec", [hlc.HLC_FP64, hlc.HLC_FP32_GUARD])
def test_output_order_fallbacks(prec):
    """Row ordering when the id buckets do not apply: one A source matched by
    3000 B sources (a bucket larger than shared memory), and all A ids equal."""
    rng = np.random.default_rng(5)
    nb = 3000
    ra_b = 10.0 + rng.uniform(-1, 1, nb) * 0.3 / 3600
    dec_b = 20.0 + rng.uniform(-1, 1, nb) * 0.3 / 3600
    idb = rng.integers(0, 2 ** 63, nb).astype(np.uint64)
    ra_a = np.concatenate([[10.0], rng.uniform(0, 360, 2000)])
    dec_a = np.concatenate([[20.0], rng.uniform(-60, 60, 2000)])
    ida = rng.integers(0, 2 ** 63, ra_a.size).astype(np.uint64)
    want, st = _check((ra_a, dec_a, ida), (ra_b, dec_b, idb), 1.0, 12, hlc.HLC_COMPLETE8, prec)
    assert want["id_a"].size >= nb
    same = np.full(ra_a.size, 12345, dtype=np.uint64)
    _check((ra_a, dec_a, same), (ra_b, dec_b, idb), 1.0, 12, hlc.HLC_COMPLETE8, prec)


def test_plans_in_two_threads_and_stream_ordered_result_copies():
    """Two host threads, each with its own stream, plan and match pinned host
    catalogues at the same time; the rows copied back without waiting (read
    after hlc_free, which synchronises the plan's stream) equal the oracle's."""
    import threading
    A, B = synth.fullsky_pair(na=300_000, nb=300_000)
    An, Bn = A.numpy(), B.numpy()
    want = O.match(*An, *Bn, 1.5, 12, O.COMPLETE)
    n = want["id_a"].size
    assert n > 50_000

    def pinned(X):
        return tuple(torch.as_tensor(np.asarray(v).view(np.int64) if v.dtype == np.uint64 else v)
                     .pin_memory() for v in X)
    Ah, Bh = pinned(An), pinned(Bn)
    got, errs = {}, []

    def worker(w):
        try:
            s = torch.cuda.Stream()
            outb = tuple(torch.empty(n + 16, dtype=dt).pin_memory()
                         for dt in (torch.int64, torch.int64, torch.float64))
            for it in range(3):
                plan = hlc.hlc_plan(Ah, Bh, 1.5, 12, precision=hlc.HLC_FP32_GUARD, stream=s)
                hlc.hlc_match(plan, copy=False)
                ia, ib, sp = hlc.hlc_result_to_host(plan, out=outb, wait=False)
                hlc.hlc_free(plan)  # (synchronises the plan's stream: the copies are done)
                got[(w, it)] = (ia.copy(), ib.copy(), sp.copy())
        except Exception as e:  # noqa: BLE001 (reported below)
            errs.append(e)
    ths = [threading.Thread(target=worker, args=(w,)) for w in range(2)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert not errs, errs
    assert len(got) == 6
    for ia, ib, sp in got.values():
        np.testing.assert_array_equal(ia, want["id_a"])
        np.testing.assert_array_equal(ib, want["id_b"])
        assert np.max(np.abs(sp - want["sep"])) <= SEP_TOL


def _clumped_pair(ks, seed, n_background=3000):
    """A: one source per clump plus a sparse background; B: k sources within
    0.3 arcsec of clump i's A source for k = ks[i], so that the A source's id
    is matched exactly k times (an output bucket of at least k rows)."""
    rng = np.random.default_rng(seed)
    ra_a = [15.0 + 3.0 * i for i in range(len(ks))]
    dec_a = [-10.0 + 2.0 * i for i in range(len(ks))]
    ra_b, dec_b = [], []
    for i, k in enumerate(ks):
        ra_b.append(ra_a[i] + rng.uniform(-1, 1, k) * 0.3 / 3600)
        dec_b.append(dec_a[i] + rng.uniform(-1, 1, k) * 0.3 / 3600)
    ra_a = np.concatenate([ra_a, rng.uniform(0, 360, n_background)])
    dec_a = np.concatenate([dec_a, rng.uniform(-60, 60, n_background)])
    ra_b = np.concatenate(ra_b + [rng.uniform(0, 360, n_background)])
    dec_b = np.concatenate(dec_b + [rng.uniform(-60, 60, n_background)])
    ida = rng.integers(0, 2 ** 63, ra_a.size).astype(np.uint64)
    idb = rng.integers(0, 2 ** 63, ra_b.size).astype(np.uint64)
    return (ra_a, dec_a, ida), (ra_b, dec_b, idb)


@pytest.mark.parametrize("prec", [hlc.HLC_FP64, hlc.HLC_FP32_GUARD])
def test_output_bucket_size_classes(prec):
    """Buckets ordered by rank counting (<= 32 rows), by the small-array
    bitonic sort (33-256), by the large one (257-2048) and by the radix
    fallback (3000 rows for one id) give the oracle's rows in order."""
    ks = [40, 200, 300, 1500]
    A, B = _clumped_pair(ks, seed=21)
    want, st = _check(A, B, 1.0, 12, hlc.HLC_COMPLETE8, prec)
    for i, k in enumerate(ks):
        assert np.count_nonzero(want["id_a"] == A[2][i]) == k
    A, B = _clumped_pair([3000, 300, 40], seed=22)
    want, st = _check(A, B, 1.0, 12, hlc.HLC_COMPLETE8, prec)
    assert np.count_nonzero(want["id_a"] == A[2][0]) == 3000
