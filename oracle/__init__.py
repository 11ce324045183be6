"""The CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, single-threaded FP64 C statement of HLC2's positional cross-match
(arXiv 2301.07331): the predicate of Eq. 1 (Sec. 2.1) in its squared-chord
form, HEALPix nested ang2pix ("hp_nestid", Sec. 4.2), the complete
8-neighbour rule and the quad-direction boundary strategy (Sec. 3.2,
Algorithm 1).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA library (``paper_2301_07331_b300``) and
imports nothing from it.

This module only marshals numpy arrays into the C library ``liboracle.so``,
which ``build()`` compiles with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hlc_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

COMPLETE = 0
QUAD = 1
QUAD_COS = 2


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -ffp-contract=off: no fused contractions)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hlc_oracle.h"))
    ):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Result(C.Structure):
    _fields_ = [("n", C.c_uint64), ("id_a", C.POINTER(C.c_uint64)),
                ("id_b", C.POINTER(C.c_uint64)), ("ia", C.POINTER(C.c_uint32)),
                ("ib", C.POINTER(C.c_uint32)), ("sep", C.POINTER(C.c_double)),
                ("chord2", C.POINTER(C.c_double)), ("pair_tests", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, u64, i32, u32 = C.c_double, C.c_uint64, C.c_int, C.c_uint32
        P = C.c_void_p
        L.orc_sincos_deg_n.argtypes = [P, u64, P, P]
        L.orc_norm_ra_n.argtypes = [P, u64, P]
        L.orc_unitvec_n.argtypes = [P, P, u64, P]
        L.orc_ang2pix_n.argtypes = [P, P, u64, i32, P]
        L.orc_neighbours_n.argtypes = [P, u64, i32, P]
        L.orc_pix2ang_n.argtypes = [P, u64, i32, P, P]
        L.orc_quad_cells_n.argtypes = [P, P, u64, d, i32, P, P]
        L.orc_quad_cells_mode_n.argtypes = [P, P, u64, d, i32, i32, P, P]
        L.orc_chord2_n.argtypes = [P, P, u64, P]
        L.orc_threshold.argtypes = [d]
        L.orc_threshold.restype = d
        L.orc_sep_arcsec.argtypes = [d]
        L.orc_sep_arcsec.restype = d
        L.orc_complete_max_radius.argtypes = [i32]
        L.orc_complete_max_radius.restype = d
        L.orc_coefficients.argtypes = [P, P]
        L.orc_match.argtypes = [P, P, P, u64, P, P, P, u64, d, i32, i32,
                                C.POINTER(_Result)]
        L.orc_match.restype = i32
        L.orc_match_brute.argtypes = [P, P, P, u64, P, P, P, u64, d,
                                      C.POINTER(_Result)]
        L.orc_match_brute.restype = i32
        L.orc_result_free.argtypes = [C.POINTER(_Result)]
        L.orc_match_eq4.argtypes = [P, P, P, P, u64, P, P, P, P, u64, i32, C.POINTER(_Result)]
        L.orc_match_eq4.restype = i32
        L.orc_match_brute_eq4.argtypes = [P, P, P, P, u64, P, P, P, P, u64,
                                          C.POINTER(_Result)]
        L.orc_match_brute_eq4.restype = i32
        L.orc_pair_radius.argtypes = [d, d]
        L.orc_pair_radius.restype = d
        L.orc_pair_radius_n.argtypes = [P, P, u64, P]
        _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _u64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def coefficients():
    s = np.zeros(10)
    c = np.zeros(11)
    lib().orc_coefficients(_p(s), _p(c))
    return s, c


def sincos_deg(x):
    x = _f64(x)
    s = np.empty_like(x)
    c = np.empty_like(x)
    lib().orc_sincos_deg_n(_p(x), x.size, _p(s), _p(c))
    return s, c


def norm_ra(ra):
    ra = _f64(ra)
    out = np.empty_like(ra)
    lib().orc_norm_ra_n(_p(ra), ra.size, _p(out))
    return out


def unitvec(ra, dec):
    ra, dec = _f64(ra), _f64(dec)
    v = np.empty((ra.size, 3))
    lib().orc_unitvec_n(_p(ra), _p(dec), ra.size, _p(v))
    return v


def chord2(va, vb):
    va, vb = _f64(va).reshape(-1, 3), _f64(vb).reshape(-1, 3)
    out = np.empty(va.shape[0])
    lib().orc_chord2_n(_p(va), _p(vb), va.shape[0], _p(out))
    return out


def threshold(r_arcsec: float) -> float:
    return lib().orc_threshold(float(r_arcsec))


def sep_arcsec(c2: float) -> float:
    return lib().orc_sep_arcsec(float(c2))


def complete_max_radius(order: int) -> float:
    return lib().orc_complete_max_radius(int(order))


def ang2pix(ra, dec, order: int):
    ra, dec = _f64(ra), _f64(dec)
    out = np.empty(ra.size, dtype=np.uint64)
    lib().orc_ang2pix_n(_p(ra), _p(dec), ra.size, int(order), _p(out))
    return out


def neighbours(pix, order: int):
    pix = _u64(pix)
    out = np.empty((pix.size, 8), dtype=np.int64)
    lib().orc_neighbours_n(_p(pix), pix.size, int(order), _p(out))
    return out


def pix2ang(pix, order: int):
    pix = _u64(pix)
    ra = np.empty(pix.size)
    dec = np.empty(pix.size)
    lib().orc_pix2ang_n(_p(pix), pix.size, int(order), _p(ra), _p(dec))
    return ra, dec


def quad_cells(ra, dec, r_arcsec: float, order: int, cosdec: bool = False):
    """Quad-direction cells (Algorithm 1); cosdec: the RA shift R / cos(dec)."""
    ra, dec = _f64(ra), _f64(dec)
    out = np.empty((ra.size, 5), dtype=np.uint64)
    cnt = np.empty(ra.size, dtype=np.int32)
    lib().orc_quad_cells_mode_n(_p(ra), _p(dec), ra.size, float(r_arcsec), int(order),
                                int(bool(cosdec)), _p(out), _p(cnt))
    return out, cnt


class OracleError(RuntimeError):
    pass


def _collect(res: _Result) -> dict:
    n = res.n
    def arr(ptr, dt):
        if n == 0:
            return np.empty(0, dtype=dt)
        return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True)
    out = dict(id_a=arr(res.id_a, np.uint64), id_b=arr(res.id_b, np.uint64),
               ia=arr(res.ia, np.uint32), ib=arr(res.ib, np.uint32),
               sep=arr(res.sep, np.float64), chord2=arr(res.chord2, np.float64),
               pair_tests=int(res.pair_tests))
    lib().orc_result_free(C.byref(res))
    return out


def match(ra_a, dec_a, id_a, ra_b, dec_b, id_b, r_arcsec: float, order: int,
          mode: int = COMPLETE) -> dict:
    """Every (A_i, B_j) with separation <= r (complete) or the quad-direction
    set (quad).  Returns arrays sorted by (id_a, id_b), ties by (ia, ib)."""
    ra_a, dec_a, id_a = _f64(ra_a), _f64(dec_a), _u64(id_a)
    ra_b, dec_b, id_b = _f64(ra_b), _f64(dec_b), _u64(id_b)
    res = _Result()
    rc = lib().orc_match(_p(ra_a), _p(dec_a), _p(id_a), ra_a.size, _p(ra_b),
                         _p(dec_b), _p(id_b), ra_b.size, float(r_arcsec),
                         int(order), int(mode), C.byref(res))
    if rc != 0:
        raise OracleError("orc_match failed with code %d" % rc)
    return _collect(res)


def match_brute(ra_a, dec_a, id_a, ra_b, dec_b, id_b, r_arcsec: float) -> dict:
    ra_a, dec_a, id_a = _f64(ra_a), _f64(dec_a), _u64(id_a)
    ra_b, dec_b, id_b = _f64(ra_b), _f64(dec_b), _u64(id_b)
    res = _Result()
    rc = lib().orc_match_brute(_p(ra_a), _p(dec_a), _p(id_a), ra_a.size,
                               _p(ra_b), _p(dec_b), _p(id_b), ra_b.size,
                               float(r_arcsec), C.byref(res))
    if rc != 0:
        raise OracleError("orc_match_brute failed with code %d" % rc)
    return _collect(res)


def pair_radius(e1, e2):
    """Eq. 4 pair radius 3 sqrt(e1^2 + e2^2) (arcsec), element-wise."""
    e1, e2 = np.broadcast_arrays(_f64(e1), _f64(e2))
    e1, e2 = _f64(e1), _f64(e2)
    out = np.empty(e1.shape)
    lib().orc_pair_radius_n(_p(e1), _p(e2), e1.size, _p(out))
    return out


def match_eq4(ra_a, dec_a, id_a, err_a, ra_b, dec_b, id_b, err_b, order: int) -> dict:
    """Complete-mode match with per-source error radii (Eq. 4): every
    (A_i, B_j) with separation <= 3 sqrt(err_a[i]^2 + err_b[j]^2) arcsec."""
    ra_a, dec_a, id_a, err_a = _f64(ra_a), _f64(dec_a), _u64(id_a), _f64(err_a)
    ra_b, dec_b, id_b, err_b = _f64(ra_b), _f64(dec_b), _u64(id_b), _f64(err_b)
    res = _Result()
    rc = lib().orc_match_eq4(_p(ra_a), _p(dec_a), _p(id_a), _p(err_a), ra_a.size, _p(ra_b),
                             _p(dec_b), _p(id_b), _p(err_b), ra_b.size, int(order),
                             C.byref(res))
    if rc != 0:
        raise OracleError("orc_match_eq4 failed with code %d" % rc)
    return _collect(res)


def match_brute_eq4(ra_a, dec_a, id_a, err_a, ra_b, dec_b, id_b, err_b) -> dict:
    ra_a, dec_a, id_a, err_a = _f64(ra_a), _f64(dec_a), _u64(id_a), _f64(err_a)
    ra_b, dec_b, id_b, err_b = _f64(ra_b), _f64(dec_b), _u64(id_b), _f64(err_b)
    res = _Result()
    rc = lib().orc_match_brute_eq4(_p(ra_a), _p(dec_a), _p(id_a), _p(err_a), ra_a.size,
                                   _p(ra_b), _p(dec_b), _p(id_b), _p(err_b), ra_b.size,
                                   C.byref(res))
    if rc != 0:
        raise OracleError("orc_match_brute_eq4 failed with code %d" % rc)
    return _collect(res)
