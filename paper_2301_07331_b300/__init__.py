"""Python binding of the B300 positional cross-match library (libhlc.so).

Argument marshalling only: every step of the match runs in the library's
CUDA kernels.  PyTorch provides device memory (the library allocates through
torch's caching allocator via a callback) and streams.  The binding refuses to
run without the compiled library or without a CUDA device; there is no CPU
fallback.

Names follow the C ABI in include/hlc.h: hlc_plan, hlc_match, hlc_free,
hlc_ang2pix, hlc_neighbours, hlc_quad_cells, hlc_unitvec, hlc_sort_pairs,
hlc_cell_table, hlc_learned_lookup.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libhlc.so")

HLC_OK, HLC_EINVAL, HLC_ENOMEM, HLC_ECUDA, HLC_ETIMEOUT, HLC_EUNSUPPORTED = range(6)
HLC_COMPLETE8, HLC_QUAD, HLC_QUAD_COSDEC = 0, 1, 2
HLC_FP64, HLC_FP32_GUARD = 0, 1
HLC_INDEX_BSEARCH, HLC_INDEX_LEARNED = 0, 1
HLC_MODEL_PLA, HLC_MODEL_MLP, HLC_MODEL_NONE = 0, 1, 2
HLC_RADIUS_FIXED, HLC_RADIUS_EQ4 = 0, 1

_ERRNAMES = {1: "HLC_EINVAL", 2: "HLC_ENOMEM", 3: "HLC_ECUDA", 4: "HLC_ETIMEOUT",
             5: "HLC_EUNSUPPORTED"}


class HLCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, str(code)), msg))
        self.code = code


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_DEALLOC_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_NO_ALLOC = _ALLOC_FN()      # NULL callbacks: the library's stream-ordered pool
_NO_DEALLOC = _DEALLOC_FN()


class Catalog(C.Structure):
    _fields_ = [("ra_deg", C.c_void_p), ("dec_deg", C.c_void_p), ("id", C.c_void_p),
                ("n", C.c_uint64), ("on_device", C.c_int), ("err_arcsec", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("radius_arcsec", C.c_double), ("coarse_level", C.c_int),
                ("fine_level", C.c_int), ("boundary", C.c_int), ("precision", C.c_int),
                ("index", C.c_int), ("model", C.c_int), ("want_sep", C.c_int),
                ("device_mem_budget", C.c_uint64), ("stream", C.c_void_p),
                ("alloc", _ALLOC_FN), ("dealloc", _DEALLOC_FN), ("alloc_ctx", C.c_void_p),
                ("tune", C.c_void_p), ("radius_rule", C.c_int)]


class TransferFit(C.Structure):
    """hlc_transfer_fit: alpha and beta of Eq. 5 per direction."""
    _fields_ = [("alpha_s", C.c_double * 2), ("beta_s_per_byte", C.c_double * 2),
                ("gbs", C.c_double * 2), ("check_bytes", C.c_uint64 * 4),
                ("check_measured_s", (C.c_double * 4) * 2), ("check_model_s", (C.c_double * 4) * 2)]


class Tune(C.Structure):
    """hlc_tune: the batched form's order target and tile shape."""
    _fields_ = [("target_per_cell", C.c_double), ("ka", C.c_uint32 * 3), ("stage", C.c_uint32)]

    def as_dict(self) -> dict:
        return {"target_per_cell": self.target_per_cell, "ka": list(self.ka),
                "stage": self.stage}


class TuneTrial(C.Structure):
    _fields_ = [("tune", Tune), ("ms", C.c_float)]


class TuneReport(C.Structure):
    _fields_ = [("best", Tune), ("ms_rule", C.c_float), ("ms_best", C.c_float),
                ("sample_jobs", C.c_uint32), ("n_trials", C.c_uint32),
                ("trials", TuneTrial * 32)]


class Result(C.Structure):
    _fields_ = [("n", C.c_uint64), ("id_a", C.c_void_p), ("id_b", C.c_void_p),
                ("sep_arcsec", C.c_void_p), ("job", C.c_void_p), ("on_device", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_a", C.c_uint64), ("n_b", C.c_uint64), ("entries_a", C.c_uint64),
                ("entries_b", C.c_uint64), ("cells_a", C.c_uint64), ("cells_b", C.c_uint64),
                ("pair_tests", C.c_uint64), ("band_candidates", C.c_uint64),
                ("matches", C.c_uint64), ("quad_duplicates", C.c_uint64),
                ("partitions", C.c_uint64), ("learned_models", C.c_uint64),
                ("learned_hit_rate", C.c_double), ("learned_max_err", C.c_uint32),
                ("join_level", C.c_int)] + [
                (f, C.c_float) for f in ("ms_prep", "ms_sort", "ms_index", "ms_candidates",
                                          "ms_pair", "ms_recheck", "ms_output", "ms_h2d",
                                          "ms_d2h", "ms_total")] + [
                ("kernel_launches", C.c_uint64), ("dense_entries_b", C.c_uint64),
                ("tile_items", C.c_uint64), ("tile_entries_a", C.c_uint64)] + [
                (f, C.c_float) for f in ("ms_stream_count", "ms_stream_bucket",
                                          "ms_stream_groups", "ms_stream_merge",
                                          "ms_sort_passes")] + [("sort_passes", C.c_uint32),
                                                                ("band_fp64", C.c_uint64),
                                                                ("sort_entries", C.c_uint64),
                                                                ("ms_plan_span", C.c_float)] + [
                (f, C.c_uint64) for f in ("h2d_bytes", "h2d_copies", "d2h_bytes",
                                          "d2h_copies")] + [
                ("ms_model_h2d", C.c_float), ("ms_model_d2h", C.c_float),
                ("stream_chunk", C.c_uint64), ("ms_tile", C.c_float), ("tile_tests", C.c_uint64),
                ("ms_plan_presort", C.c_float), ("sort_bytes", C.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _SO


def lib():
    """Load libhlc.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(_SO):
        raise RuntimeError("libhlc.so is missing; run paper_2301_07331_b300/build.py")
    L = C.CDLL(_SO)
    P, u64, i32, d = C.c_void_p, C.c_uint64, C.c_int, C.c_double
    L.hlc_plan.argtypes = [P, P, P, C.c_uint32, C.POINTER(C.c_void_p)]
    L.hlc_match.argtypes = [P, C.POINTER(Result), P]
    L.hlc_free.argtypes = [P]
    L.hlc_free.restype = None
    L.hlc_result_to_host.argtypes = [P, P, P, P, P]
    L.hlc_result_to_host_async.argtypes = [P, P, P, P, P, P]
    L.hlc_last_error.restype = C.c_char_p
    L.hlc_version.restype = C.c_char_p
    L.hlc_abi_sizes.argtypes = [C.POINTER(C.c_size_t), C.c_int]
    L.hlc_abi_sizes.restype = C.c_int
    L.hlc_canonical_coefficients.argtypes = [P, P]
    L.hlc_ang2pix.argtypes = [P, P, u64, i32, i32, P, P]
    L.hlc_neighbours.argtypes = [P, u64, i32, P, P]
    L.hlc_quad_cells.argtypes = [P, P, u64, d, i32, i32, i32, P, P, P]
    L.hlc_unitvec.argtypes = [P, P, u64, P, P]
    L.hlc_sort_pairs.argtypes = [P, P, u64, i32, i32, P]
    L.hlc_sort_pairs_noalloc.argtypes = [P, P, u64, i32, i32, P]
    L.hlc_cell_table.argtypes = [P, u64, P, P, C.POINTER(C.c_uint64), P]
    L.hlc_learned_lookup.argtypes = [P, u64, i32, i32, P, u64, P, P, P]
    L.hlc_autotune.argtypes = [P, P, P, C.c_uint32, C.c_uint32, P]
    L.hlc_transfer_model.argtypes = [P]
    L.hlc_test_spin_shift.argtypes = [i32]
    L.hlc_test_unset_wait.argtypes = [i32, P]
    _lib = L
    return L


def _check(rc: int):
    if rc != HLC_OK:
        raise HLCError(rc, lib().hlc_last_error().decode(errors="replace"))


_cuda_seen = False


def _require_cuda():
    global _cuda_seen
    if _cuda_seen:
        return
    if not torch.cuda.is_available():
        raise RuntimeError("the cross-match library needs a CUDA device (none visible)")
    _cuda_seen = True


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t: torch.Tensor) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def version() -> str:
    return lib().hlc_version().decode()


def hlc_canonical_coefficients():
    s = np.zeros(10)
    c = np.zeros(11)
    _check(lib().hlc_canonical_coefficients(s.ctypes.data, c.ctypes.data))
    return s, c


# ---------------------------------------------------------------------------
# Allocation through torch's caching allocator.
# ---------------------------------------------------------------------------
class _TorchAllocator:
    def __init__(self, device: int, stream: int):
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, ctx):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def _dealloc(ptr, ctx):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = _ALLOC_FN(_alloc)
        self.dealloc = _DEALLOC_FN(_dealloc)


@dataclass
class Plan:
    handle: C.c_void_p
    params: Params
    allocator: object
    keep: tuple
    result: Result | None = None

    def __del__(self):
        try:
            hlc_free(self)
        except Exception:
            pass


def _catalog(ra, dec, ids, err=None):
    """Catalog struct for torch (CUDA or CPU) tensors or numpy arrays; err:
    optional per-source error radii (arcsec) in the same memory space."""
    if isinstance(ra, torch.Tensor):
        on_dev = ra.is_cuda
        ra = ra.contiguous().to(torch.float64)
        dec = dec.contiguous().to(torch.float64)
        ids = ids.contiguous()
        if ids.dtype not in (torch.int64, torch.uint64):
            ids = ids.to(torch.int64)
        if err is not None:
            err = torch.as_tensor(err, dtype=torch.float64, device=ra.device).contiguous()
        if not on_dev:
            ptrs = (ra.data_ptr(), dec.data_ptr(), ids.data_ptr(),
                    err.data_ptr() if err is not None else None)
        else:
            ptrs = (_dptr(ra), _dptr(dec), _dptr(ids), _dptr(err) if err is not None else None)
        return (Catalog(ptrs[0], ptrs[1], ptrs[2], ra.numel(), int(on_dev), ptrs[3]),
                (ra, dec, ids, err))
    ra = np.ascontiguousarray(ra, dtype=np.float64)
    dec = np.ascontiguousarray(dec, dtype=np.float64)
    ids = np.ascontiguousarray(ids).view(np.uint64) if np.asarray(ids).dtype.itemsize == 8 \
        else np.ascontiguousarray(ids, dtype=np.uint64)
    if err is not None:
        err = np.ascontiguousarray(err, dtype=np.float64)
    return (Catalog(ra.ctypes.data, dec.ctypes.data, ids.ctypes.data, ra.size, 0,
                    err.ctypes.data if err is not None else None), (ra, dec, ids, err))


def hlc_plan(A, B, radius_arcsec: float, fine_level: int, coarse_level: int | None = None,
             boundary: int = HLC_COMPLETE8, precision: int = HLC_FP32_GUARD,
             index: int = HLC_INDEX_BSEARCH, model: int = HLC_MODEL_PLA, want_sep: bool = True,
             device_mem_budget: int = 0, stream=None, torch_alloc: bool = False,
             err_a=None, err_b=None) -> Plan:
    """Index two catalogues.  A and B are (ra, dec, id) triples (torch tensors
    on the device or host, or numpy arrays on the host) or objects with .ra,
    .dec, .id.  Device memory comes from the library's stream-ordered pool,
    or from torch's caching allocator with torch_alloc=True.  With err_a and
    err_b (per-source error radii in arcsec, beside the coordinates) the
    radius of each pair is Eq. 4's 3 sqrt(err_a[i]^2 + err_b[j]^2) and
    radius_arcsec is ignored.  Returns a Plan for hlc_match."""
    _require_cuda()
    L = lib()
    if (err_a is None) != (err_b is None):
        raise ValueError("give both err_a and err_b (Eq. 4) or neither")
    cA, keepA = _catalog(*(_triple(A)), err=err_a)
    cB, keepB = _catalog(*(_triple(B)), err=err_b)
    st = _stream_ptr(stream)
    alloc = _TorchAllocator(torch.cuda.current_device(), st) if torch_alloc else None
    p = Params(float(radius_arcsec), int(fine_level if coarse_level is None else coarse_level),
               int(fine_level), int(boundary), int(precision), int(index), int(model),
               int(bool(want_sep)), int(device_mem_budget), st,
               alloc.alloc if alloc else _NO_ALLOC, alloc.dealloc if alloc else _NO_DEALLOC,
               None)
    if coarse_level is None:
        p.coarse_level = min(4, int(fine_level))
    p.radius_rule = HLC_RADIUS_EQ4 if err_a is not None else HLC_RADIUS_FIXED
    h = C.c_void_p()
    _check(L.hlc_plan(C.byref(cA), C.byref(cB), C.byref(p), 1, C.byref(h)))
    return Plan(h, p, alloc, (keepA, keepB))


def _batched_args(jobs, precision, want_sep, stream, torch_alloc, tune):
    n = len(jobs)
    cats_a = (Catalog * n)()
    cats_b = (Catalog * n)()
    params = (Params * n)()
    keep = []
    st = _stream_ptr(stream)
    dev = torch.cuda.current_device()
    alloc = _TorchAllocator(dev, st) if torch_alloc else None
    for i, jb in enumerate(jobs):
        ca, ka = _catalog(*_triple(jb["A"]))
        cb, kb = _catalog(*_triple(jb["B"]))
        cats_a[i] = ca
        cats_b[i] = cb
        keep.append((ka, kb))
        fl = int(jb.get("fine_level", -1))
        params[i] = Params(float(jb["radius_arcsec"]), 0, fl, HLC_COMPLETE8, int(precision),
                           HLC_INDEX_BSEARCH, HLC_MODEL_PLA, int(bool(want_sep)), 0, st,
                           alloc.alloc if alloc else _NO_ALLOC,
                           alloc.dealloc if alloc else _NO_DEALLOC, None,
                           C.addressof(tune) if tune is not None else None, HLC_RADIUS_FIXED)
    return n, cats_a, cats_b, params, keep, alloc


def hlc_transfer_model() -> dict:
    """Measure the transfer-cost model of Eq. 5 (alpha, beta per direction)."""
    _require_cuda()
    f = TransferFit()
    _check(lib().hlc_transfer_model(C.byref(f)))
    names = ("h2d", "d2h")
    out = {}
    for k, nm in enumerate(names):
        out[nm] = {"alpha_s": f.alpha_s[k], "beta_s_per_byte": f.beta_s_per_byte[k],
                   "gbs": f.gbs[k],
                   "check": [{"bytes": int(f.check_bytes[i]),
                              "measured_s": f.check_measured_s[k][i],
                              "model_s": f.check_model_s[k][i]} for i in range(4)]}
    return out


def hlc_autotune(jobs, sample_jobs: int = 256, precision: int = HLC_FP32_GUARD, stream=None):
    """Time the batched form's candidate order targets and tile shapes on a
    sample of these jobs (same job dicts as hlc_plan_batched).  Returns the
    best Tune (to pass as hlc_plan_batched(..., tune=)) and the report."""
    _require_cuda()
    n, ca, cb, params, keep, _ = _batched_args(jobs, precision, True, stream, False, None)
    rep = TuneReport()
    _check(lib().hlc_autotune(ca, cb, params, n, int(sample_jobs), C.byref(rep)))
    best = Tune()
    C.pointer(best)[0] = rep.best
    trials = [dict(rep.trials[i].tune.as_dict(), ms=rep.trials[i].ms)
              for i in range(rep.n_trials)]
    return best, {"best": rep.best.as_dict(), "ms_rule": rep.ms_rule, "ms_best": rep.ms_best,
                  "sample_jobs": rep.sample_jobs, "trials": trials}


class BatchedJobs:
    """A job list marshalled once into the C structs hlc_plan takes (what a C
    caller builds once), for plans over the same catalogue buffers again and
    again: building them costs about 10 us a job in Python.  The tensors must
    stay alive and unchanged in place while plans are made from it."""

    def __init__(self, jobs, precision: int = HLC_FP32_GUARD, want_sep: bool = True,
                 stream=None, torch_alloc: bool = False, tune: Tune | None = None):
        _require_cuda()
        (self.n, self.cats_a, self.cats_b, self.params, self.keep,
         self.alloc) = _batched_args(jobs, precision, want_sep, stream, torch_alloc, tune)
        self.tune = tune


def hlc_plan_batched(jobs, precision: int = HLC_FP32_GUARD, want_sep: bool = True,
                     stream=None, torch_alloc: bool = False, tune: Tune | None = None) -> Plan:
    """One plan over many independent jobs.  jobs: sequence of dicts with keys
    A, B ((ra, dec, id) triples or catalogue objects), radius_arcsec and
    fine_level (-1 = chosen by the library from the job's density), or a
    BatchedJobs (which carries its own precision, stream and tune; the other
    arguments are then ignored).  tune: a Tune from hlc_autotune (None: the
    library's rule)."""
    _require_cuda()
    L = lib()
    if not isinstance(jobs, BatchedJobs):
        jobs = BatchedJobs(jobs, precision, want_sep, stream, torch_alloc, tune)
    h = C.c_void_p()
    _check(L.hlc_plan(jobs.cats_a, jobs.cats_b, jobs.params, jobs.n, C.byref(h)))
    return Plan(h, jobs.params[0], jobs.alloc, (jobs.keep, jobs.cats_a, jobs.cats_b, jobs.params,
                                                jobs.tune))


def _triple(X):
    if isinstance(X, (tuple, list)):
        return X
    return X.ra, X.dec, X.id


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr or 0, False), "version": 3}


def _as_tensor(ptr, n, typestr, dtype, copy):
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    t = torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")
    return t.clone() if copy else t


def hlc_match(plan: Plan, copy: bool = True) -> dict:
    """Run the match.  Returns id_a, id_b (int64 bit patterns of the uint64
    ids), sep (float64 arcsec or None) as CUDA tensors, and the stats dict.
    With copy=False the tensors alias the plan's memory (valid until
    hlc_free or the next hlc_match)."""
    L = lib()
    r = Result()
    s = Stats()
    _check(L.hlc_match(plan.handle, C.byref(r), C.byref(s)))
    plan.result = r
    n = int(r.n)
    if not r.on_device:  # streamed plans return host rows
        def host(ptr, ct, dt):
            if n == 0 or not ptr:
                return torch.empty(0, dtype=dt)
            a = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(n,))
            if copy:  # else a view of the plan's pinned rows (valid until hlc_free)
                a = a.copy()
            return torch.from_numpy(a.view(np.int64) if dt == torch.int64 else a)
        return dict(n=n, id_a=host(r.id_a, C.c_uint64, torch.int64),
                    id_b=host(r.id_b, C.c_uint64, torch.int64),
                    sep=host(r.sep_arcsec, C.c_double, torch.float64) if r.sep_arcsec else None,
                    job=None, stats=s.as_dict())
    return dict(n=n,
                id_a=_as_tensor(r.id_a, n, "<i8", torch.int64, copy),
                id_b=_as_tensor(r.id_b, n, "<i8", torch.int64, copy),
                sep=_as_tensor(r.sep_arcsec, n, "<f8", torch.float64, copy)
                if r.sep_arcsec else None,
                job=_as_tensor(r.job, n, "<u4", torch.int32, copy) if r.job else None,
                stats=s.as_dict())


def hlc_result_to_host(plan: Plan, out=None, wait: bool = True):
    """Copy the last result's rows to host memory.  out: optional (id_a, id_b,
    sep) host buffers (numpy arrays or CPU tensors, pinned ones copy fastest)
    with room for n rows; the returned arrays are views of their first n.
    wait=False enqueues the copies on the plan's stream and returns at once
    (read the arrays after synchronising that stream, or after hlc_free of
    the plan, which does)."""
    r = plan.result
    n = int(r.n)

    def buf(i, dt):
        if out is None:
            return np.empty(n, dt)
        b = out[i]
        b = b.numpy() if isinstance(b, torch.Tensor) else b
        if b.size < n:
            raise ValueError("output buffer %d holds %d rows, %d needed" % (i, b.size, n))
        return b[:n].view(dt)
    ia, ib = buf(0, np.uint64), buf(1, np.uint64)
    sp = buf(2, np.float64) if r.sep_arcsec else None
    sp_ptr = sp.ctypes.data if sp is not None else None
    if wait:
        _check(lib().hlc_result_to_host(C.byref(r), ia.ctypes.data, ib.ctypes.data, sp_ptr, None))
    else:
        _check(lib().hlc_result_to_host_async(C.byref(r), ia.ctypes.data, ib.ctypes.data, sp_ptr,
                                              None, plan.params.stream))
    return ia, ib, sp


def hlc_free(plan: Plan):
    if plan is not None and plan.handle:
        lib().hlc_free(plan.handle)
        plan.handle = C.c_void_p()


# ---------------------------------------------------------------------------
# Kernel-level entry points.
# ---------------------------------------------------------------------------
def hlc_ang2pix(ra: torch.Tensor, dec: torch.Tensor, order: int, precision: int = HLC_FP64,
                stream=None) -> torch.Tensor:
    """Nested pixel ids (int32 tensor holding uint32 values)."""
    _require_cuda()
    out = torch.empty(ra.numel(), dtype=torch.int32, device=ra.device)
    _check(lib().hlc_ang2pix(_dptr(ra), _dptr(dec), ra.numel(), int(order), int(precision),
                             _dptr(out) if out.numel() else None, _stream_ptr(stream)))
    return out


def hlc_neighbours(pix: torch.Tensor, order: int, stream=None) -> torch.Tensor:
    _require_cuda()
    out = torch.empty((pix.numel(), 8), dtype=torch.int64, device=pix.device)
    _check(lib().hlc_neighbours(_dptr(pix), pix.numel(), int(order),
                                _dptr(out) if out.numel() else None, _stream_ptr(stream)))
    return out


def hlc_quad_cells(ra, dec, radius_arcsec: float, order: int, precision: int = HLC_FP64,
                   stream=None, boundary: int = HLC_QUAD):
    _require_cuda()
    out = torch.empty((ra.numel(), 5), dtype=torch.int32, device=ra.device)
    cnt = torch.empty(ra.numel(), dtype=torch.int32, device=ra.device)
    _check(lib().hlc_quad_cells(_dptr(ra), _dptr(dec), ra.numel(), float(radius_arcsec),
                                int(order), int(precision), int(boundary),
                                _dptr(out) if out.numel() else None,
                                _dptr(cnt) if cnt.numel() else None, _stream_ptr(stream)))
    return out, cnt


def hlc_unitvec(ra, dec, stream=None) -> torch.Tensor:
    _require_cuda()
    out = torch.empty((ra.numel(), 3), dtype=torch.float64, device=ra.device)
    _check(lib().hlc_unitvec(_dptr(ra), _dptr(dec), ra.numel(),
                             _dptr(out) if out.numel() else None, _stream_ptr(stream)))
    return out


def hlc_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, key_bits: int, stream=None):
    """In-place stable radix sort of (keys, vals); keys int32/int64 bit
    patterns of unsigned keys, vals int32 bit patterns of uint32."""
    _require_cuda()
    ks = keys.element_size()
    _check(lib().hlc_sort_pairs(_dptr(keys), _dptr(vals), keys.numel(), ks, int(key_bits),
                                _stream_ptr(stream)))
    return keys, vals


def hlc_sort_pairs_noalloc(keys: torch.Tensor, vals: torch.Tensor, key_bits: int, stream=None):
    """Same sort as hlc_sort_pairs without any device allocation: for callers
    that must not allocate on the call path (all temporaries come from a fixed
    array inside the library; at most 1,048,576 elements; concurrent calls
    race)."""
    _require_cuda()
    ks = keys.element_size()
    _check(lib().hlc_sort_pairs_noalloc(_dptr(keys), _dptr(vals), keys.numel(), ks,
                                        int(key_bits), _stream_ptr(stream)))
    return keys, vals


def hlc_cell_table(keys: torch.Tensor, stream=None):
    _require_cuda()
    n = keys.numel()
    uniq = torch.empty(max(n, 1), dtype=torch.int32, device=keys.device)
    start = torch.empty(n + 1, dtype=torch.int32, device=keys.device)
    m = C.c_uint64()
    _check(lib().hlc_cell_table(_dptr(keys) if n else None, n, _dptr(uniq), _dptr(start),
                                C.byref(m), _stream_ptr(stream)))
    m = int(m.value)
    return uniq[:m], start[:m + 1]


def hlc_learned_lookup(uniq: torch.Tensor, shift: int, model: int, queries: torch.Tensor,
                       stream=None):
    _require_cuda()
    out = torch.empty(queries.numel(), dtype=torch.int32, device=queries.device)
    s = Stats()
    _check(lib().hlc_learned_lookup(_dptr(uniq), uniq.numel(), int(shift), int(model),
                                    _dptr(queries), queries.numel(), _dptr(out), C.byref(s),
                                    _stream_ptr(stream)))
    return out, s.as_dict()
