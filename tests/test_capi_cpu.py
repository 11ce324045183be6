"""CPU-only checks of the C-ABI library: it builds, loads without a GPU,
exports every entry point include/hlc.h declares, and its binary128-derived
trigonometric constants equal the oracle's independently derived ones."""
import ctypes
import os
import re

import numpy as np

import oracle as O
import paper_2301_07331_b300 as hlc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hlc_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = hlc.lib()
    declared = _declared()
    assert {"hlc_plan", "hlc_match", "hlc_free", "hlc_last_error"} <= declared
    for name in sorted(declared):
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_binding_structs_match_the_library_layouts():
    """Every ctypes struct of the binding has the size the library was built
    with (a field added on one side only would shift the others)."""
    L = hlc.lib()
    out = (ctypes.c_size_t * 8)()
    assert L.hlc_abi_sizes(out, 8) == 8
    mine = [hlc.Catalog, hlc.Tune, hlc.TuneTrial, hlc.TuneReport, hlc.Params, hlc.Result,
            hlc.Stats, hlc.TransferFit]
    for s, cls in zip(out, mine):
        assert s == ctypes.sizeof(cls), (cls.__name__, s, ctypes.sizeof(cls))
    assert L.hlc_abi_sizes(None, 0) == 8


def test_version_and_error_string():
    assert "sm_103a" in hlc.version()
    assert hlc.lib().hlc_last_error() is not None


def test_canonical_constants_equal_oracle_bit_for_bit():
    s_lib, c_lib = hlc.hlc_canonical_coefficients()
    s_orc, c_orc = O.coefficients()
    np.testing.assert_array_equal(s_lib.view(np.uint64), s_orc.view(np.uint64))
    np.testing.assert_array_equal(c_lib.view(np.uint64), c_orc.view(np.uint64))


def test_invalid_plan_arguments_fail_before_any_device_work():
    # parameter validation happens on the host; NULL out pointer is EINVAL
    rc = hlc.lib().hlc_plan(None, None, None, 1, None)
    assert rc == hlc.HLC_EINVAL
    assert b"NULL" in hlc.lib().hlc_last_error()


def _valid_params():
    p = hlc.Params()
    p.radius_arcsec = 1.5
    p.coarse_level, p.fine_level = 4, 12
    p.boundary, p.precision = hlc.HLC_COMPLETE8, hlc.HLC_FP32_GUARD
    p.index, p.model = hlc.HLC_INDEX_BSEARCH, hlc.HLC_MODEL_PLA
    p.want_sep, p.device_mem_budget, p.stream = 1, 0, None
    p.alloc, p.dealloc, p.alloc_ctx = hlc._NO_ALLOC, hlc._NO_DEALLOC, None
    return p


def test_each_invalid_argument_is_named_before_any_device_work():
    """Every rejected argument returns HLC_EINVAL with a message naming it, and
    none of these calls reaches the device (this runs without a GPU)."""
    ra = np.array([10.0, 20.0])
    dec = np.array([-5.0, 5.0])
    ids = np.array([1, 2], dtype=np.uint64)

    def cat(n=2, null=False):
        c = hlc.Catalog()
        c.ra_deg = None if null else ra.ctypes.data
        c.dec_deg = dec.ctypes.data
        c.id = ids.ctypes.data
        c.n, c.on_device = n, 0
        return c

    def plan(p, a=None, b=None, n_jobs=1):
        out = ctypes.c_void_p()
        a = a or cat()
        b = b or cat()
        rc = hlc.lib().hlc_plan(ctypes.byref(a), ctypes.byref(b), ctypes.byref(p), n_jobs,
                                ctypes.byref(out))
        return rc, hlc.lib().hlc_last_error().decode(), out.value

    def with_(**kw):
        p = _valid_params()
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    cases = [
        (with_(radius_arcsec=0.0), "radius_arcsec"),
        (with_(radius_arcsec=-1.0), "radius_arcsec"),
        (with_(radius_arcsec=float("nan")), "radius_arcsec"),
        (with_(radius_arcsec=648000.5, boundary=hlc.HLC_QUAD), "radius_arcsec"),
        (with_(fine_level=15), "fine_level"),
        (with_(fine_level=-1), "fine_level"),
        (with_(coarse_level=13), "coarse_level"),
        (with_(coarse_level=-1), "coarse_level"),
        (with_(boundary=7), "boundary"),
        (with_(precision=5), "precision"),
        (with_(index=3), "index"),
        (with_(model=9), "model"),
        # complete mode is exact only up to theta_L / 8 (51.5 arcsec / 8 at order 12)
        (with_(radius_arcsec=10.0), "theta_L/8"),
        (with_(alloc=hlc._ALLOC_FN(lambda n, c: None)), "alloc and dealloc"),
    ]
    for p, word in cases:
        rc, msg, out = plan(p)
        assert rc == hlc.HLC_EINVAL and word in msg and not out, (word, rc, msg)
    rc, msg, _ = plan(_valid_params(), a=cat(n=1 << 31))
    assert rc == hlc.HLC_EINVAL and "2^31" in msg and "A" in msg
    rc, msg, _ = plan(_valid_params(), b=cat(null=True))
    assert rc == hlc.HLC_EINVAL and "B has NULL arrays" in msg
    rc, msg, _ = plan(_valid_params(), n_jobs=0)
    assert rc == hlc.HLC_EINVAL and "n_jobs" in msg


def test_batched_plan_and_kernel_entry_points_reject_bad_arguments_on_the_host():
    """Batched-plan consistency rules and the kernel-level entry points'
    argument checks all return before the first device call."""
    L = hlc.lib()
    ra = np.array([10.0, 20.0])
    dec = np.array([-5.0, 5.0])
    ids = np.array([1, 2], dtype=np.uint64)

    def cats(on_device=(0, 0)):
        arr = (hlc.Catalog * 2)()
        for j in range(2):
            arr[j].ra_deg, arr[j].dec_deg = ra.ctypes.data, dec.ctypes.data
            arr[j].id = ids.ctypes.data
            arr[j].n, arr[j].on_device = 2, on_device[j]
        return arr

    def batched(mod, A=None, B=None):
        ps = (hlc.Params * 2)(_valid_params(), _valid_params())
        mod(ps)
        out = ctypes.c_void_p()
        rc = L.hlc_plan(A or cats(), B or cats(), ps, 2, ctypes.byref(out))
        return rc, L.hlc_last_error().decode(), out.value

    def quad(ps):
        ps[1].boundary = hlc.HLC_QUAD

    def mixed_precision(ps):
        ps[1].precision = hlc.HLC_FP64

    def bad_radius(ps):
        ps[1].radius_arcsec = -2.0

    rc, msg, out = batched(quad)
    assert rc == hlc.HLC_EUNSUPPORTED and "complete boundary" in msg and not out
    rc, msg, out = batched(mixed_precision)
    assert rc == hlc.HLC_EINVAL and "share precision" in msg and not out
    rc, msg, out = batched(bad_radius)
    assert rc == hlc.HLC_EINVAL and "radius_arcsec" in msg and not out
    rc, msg, out = batched(lambda ps: None, A=cats((0, 1)))
    assert rc == hlc.HLC_EINVAL and "all on the host" in msg and not out

    buf = np.zeros(64, dtype=np.float64)
    p = buf.ctypes.data
    assert L.hlc_ang2pix(p, p, 4, 15, hlc.HLC_FP64, p, None) == hlc.HLC_EINVAL
    assert L.hlc_ang2pix(p, p, 4, 12, 9, p, None) == hlc.HLC_EINVAL
    assert L.hlc_ang2pix(None, p, 4, 12, hlc.HLC_FP64, p, None) == hlc.HLC_EINVAL
    assert b"NULL" in L.hlc_last_error()
    assert L.hlc_neighbours(p, 4, -1, p, None) == hlc.HLC_EINVAL
    assert L.hlc_neighbours(None, 4, 3, p, None) == hlc.HLC_EINVAL
    Q = hlc.HLC_QUAD
    assert L.hlc_quad_cells(p, p, 4, 0.0, 12, hlc.HLC_FP64, Q, p, p, None) == hlc.HLC_EINVAL
    assert L.hlc_quad_cells(p, p, 4, 1.0, 15, hlc.HLC_FP64, Q, p, p, None) == hlc.HLC_EINVAL
    assert L.hlc_quad_cells(p, p, 4, 1.0, 12, 7, Q, p, p, None) == hlc.HLC_EINVAL
    assert L.hlc_quad_cells(p, p, 4, 1.0, 12, hlc.HLC_FP64, 0, p, p, None) == hlc.HLC_EINVAL
    assert L.hlc_unitvec(p, None, 4, p, None) == hlc.HLC_EINVAL
    for ks, kb in ((2, 8), (4, 0), (4, 33), (8, 65)):
        assert L.hlc_sort_pairs(p, p, 4, ks, kb, None) == hlc.HLC_EINVAL, (ks, kb)
        assert L.hlc_sort_pairs_noalloc(p, p, 4, ks, kb, None) == hlc.HLC_EINVAL, (ks, kb)
    assert L.hlc_sort_pairs(None, p, 4, 4, 32, None) == hlc.HLC_EINVAL
    assert L.hlc_sort_pairs_noalloc(p, p, 1 << 40, 4, 32, None) == hlc.HLC_EINVAL
    assert b"use hlc_sort_pairs" in L.hlc_last_error()
    m = ctypes.c_uint64()
    assert L.hlc_cell_table(None, 4, p, p, ctypes.byref(m), None) == hlc.HLC_EINVAL
    assert L.hlc_cell_table(p, 4, p, p, None, None) == hlc.HLC_EINVAL
    assert L.hlc_learned_lookup(p, 4, 25, hlc.HLC_MODEL_PLA, p, 4, p, None, None) == \
        hlc.HLC_EINVAL
    assert L.hlc_learned_lookup(p, 4, 8, 7, p, 4, p, None, None) == hlc.HLC_EINVAL
    assert L.hlc_learned_lookup(None, 4, 8, hlc.HLC_MODEL_PLA, p, 4, p, None, None) == \
        hlc.HLC_EINVAL
    res = hlc.Result()
    assert L.hlc_match(None, ctypes.byref(res), None) == hlc.HLC_EINVAL
    assert L.hlc_result_to_host(None, p, p, p, None) == hlc.HLC_EINVAL
    assert L.hlc_canonical_coefficients(None, None) == hlc.HLC_EINVAL
    L.hlc_free(None)  # a NULL plan is a no-op
