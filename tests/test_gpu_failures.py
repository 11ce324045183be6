"""Failure paths on the GPU that fault and hang nothing.

- A device allocator callback that returns NULL on its k-th call, for every
  k the plan and the match make: HLC_ENOMEM, nothing written to the caller's
  out-parameters, every buffer handed back, and the next plan works.
- Each kind of bounded device wait run against a flag that nothing sets,
  with the poll limits shortened by the test hook: the kernel gives up,
  returns, HLC_ETIMEOUT reaches the caller and the context stays usable.
"""
import ctypes as C
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    import torch

    import paper_2301_07331_b300 as hlc
    from paper_2301_07331_b300 import synth
    torch.cuda.set_device(0)
    return torch, hlc, synth


class FailingAllocator:
    """torch's caching allocator behind the C callbacks, returning NULL on
    call number `fail_at` (1-based; 0 = never)."""

    def __init__(self, torch, hlc, fail_at):
        self.torch = torch
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}
        dev = torch.cuda.current_device()
        st = torch.cuda.current_stream().cuda_stream

        def _alloc(nbytes, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
            self.live[p] = nbytes
            return p

        def _dealloc(ptr, ctx):
            assert ptr in self.live, "freed a pointer the allocator did not hand out"
            del self.live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = hlc._ALLOC_FN(_alloc)
        self.dealloc = hlc._DEALLOC_FN(_dealloc)


def _plan_match(torch, hlc, A, B, al, precision, boundary):
    """hlc_plan + hlc_match through the raw C ABI with the given allocator.
    Returns (rc, stage, rows); the sentinels show whether out-parameters were
    written on failure."""
    L = hlc.lib()
    keep = []
    cats = []
    for X in (A, B):
        c, k = hlc._catalog(X.ra, X.dec, X.id)
        cats.append(c)
        keep.append(k)
    p = hlc.Params(1.0, 4, 13, boundary, precision, hlc.HLC_INDEX_BSEARCH, hlc.HLC_MODEL_PLA, 1, 0,
                   torch.cuda.current_stream().cuda_stream, al.alloc, al.dealloc, None)
    sentinel = C.c_void_p(0x1234)
    rc = L.hlc_plan(C.byref(cats[0]), C.byref(cats[1]), C.byref(p), 1, C.byref(sentinel))
    if rc != 0:
        assert sentinel.value == 0x1234, "hlc_plan wrote *out on failure"
        return rc, "plan", None
    res = hlc.Result(777, None, None, None, None, 5)
    rc = L.hlc_match(sentinel, C.byref(res), None)
    rows = None
    if rc != 0:
        assert res.n == 777 and res.id_a is None and res.on_device == 5, \
            "hlc_match wrote the result on failure"
    else:
        n = int(res.n)
        ia = np.empty(n, np.uint64)
        ib = np.empty(n, np.uint64)
        assert L.hlc_result_to_host(C.byref(res), ia.ctypes.data, ib.ctypes.data, None, None) == 0
        rows = (ia, ib)
    L.hlc_free(sentinel)
    return rc, "match", rows


@pytest.mark.parametrize("precision,boundary", [(1, 0), (0, 0), (1, 1)],
                         ids=["fp32_complete", "fp64_complete", "fp32_quad"])
def test_allocator_returning_null_at_every_call(precision, boundary):
    torch, hlc, synth = _setup()
    A, B = synth.patch_pair(na=6000, nb=6000)
    A, B = A.to("cuda"), B.to("cuda")
    ok = FailingAllocator(torch, hlc, 0)
    rc, _, want = _plan_match(torch, hlc, A, B, ok, precision, boundary)
    assert rc == 0 and want[0].size > 1000
    torch.cuda.synchronize()
    assert not ok.live
    total = ok.calls
    assert total >= 5
    for k in range(1, total + 1):
        al = FailingAllocator(torch, hlc, k)
        rc, stage, _ = _plan_match(torch, hlc, A, B, al, precision, boundary)
        assert rc == hlc.HLC_ENOMEM, (k, stage, rc, hlc.lib().hlc_last_error())
        torch.cuda.synchronize()
        assert not al.live, (k, stage, "buffers not handed back")
    # the device is still fine: the same match again, same rows
    rc, _, again = _plan_match(torch, hlc, A, B, FailingAllocator(torch, hlc, 0), precision,
                               boundary)
    assert rc == 0 and np.array_equal(again[0], want[0]) and np.array_equal(again[1], want[1])


@pytest.mark.parametrize("which", [0, 1, 2], ids=["sort_lookback", "scan_lookback", "mbarrier"])
def test_unset_flag_wait_times_out_and_returns(which):
    import oracle as O
    torch, hlc, synth = _setup()
    L = hlc.lib()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.hlc_test_spin_shift(16) == 0
    try:
        t0 = time.perf_counter()
        rc = L.hlc_test_unset_wait(which, stream)
        dt = time.perf_counter() - t0
        msg = L.hlc_last_error()  # (read before the next call clears it)
    finally:
        assert L.hlc_test_spin_shift(0) == 0
    assert rc == hlc.HLC_ETIMEOUT, (rc, msg)
    assert b"bounded device wait" in msg
    print("wait %d gave up after %.1f ms with the limit shifted by 16" % (which, dt * 1e3))
    # the context is usable: a match right after equals the oracle
    A, B = synth.patch_pair(na=3000, nb=3000)
    want = O.match(*A.numpy(), *B.numpy(), 1.0, 13, O.COMPLETE)
    plan = hlc.hlc_plan(A.to("cuda"), B.to("cuda"), 1.0, 13)
    res = hlc.hlc_match(plan)
    hlc.hlc_free(plan)
    assert np.array_equal(res["id_a"].cpu().numpy().view(np.uint64), want["id_a"])
    assert np.array_equal(res["id_b"].cpu().numpy().view(np.uint64), want["id_b"])


def test_spin_shift_rejects_out_of_range():
    torch, hlc, synth = _setup()
    L = hlc.lib()
    assert L.hlc_test_spin_shift(-1) == hlc.HLC_EINVAL
    assert L.hlc_test_spin_shift(25) == hlc.HLC_EINVAL
    assert L.hlc_test_unset_wait(3, None) == hlc.HLC_EINVAL
