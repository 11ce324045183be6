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
