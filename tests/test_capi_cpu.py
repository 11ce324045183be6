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
