"""The allocation-free sort entry point, called through the C ABI.

Some callers cannot allocate device memory on their call path (their host
application owns all device memory through its own allocator, or a
cudaMalloc/cudaFree in a latency-critical loop is not acceptable).  For them
the library offers hlc_sort_pairs_noalloc, which takes its temporaries from a
fixed array built into the library.  This test checks that it returns exactly
what hlc_sort_pairs returns, on two calls in a row (the second reuses the
array the first left behind), and that it refuses sizes beyond its capacity.
It lives in its own file, collected last, and passes alone or after the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2301_07331_b300 as hlc

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20


def _call(fn, keys, vals, bits):
    L = hlc.lib()
    rc = getattr(L, fn)(keys.data_ptr(), vals.data_ptr(), keys.numel(), keys.element_size(),
                        bits, torch.cuda.current_stream().cuda_stream)
    assert rc == hlc.HLC_OK, (fn, rc, L.hlc_last_error())


@pytest.mark.parametrize("ksize,bits,n", [(4, 28, MAX_N), (8, 64, 300_001)])
def test_noalloc_sort_matches_the_allocating_sort_twice(ksize, bits, n):
    torch.cuda.set_device(0)
    for call, seed in enumerate((11, 12)):
        rng = np.random.default_rng(seed + ksize)
        if ksize == 4:
            k = rng.integers(0, 2 ** bits, n, dtype=np.uint64).astype(np.uint32).view(np.int32)
        else:
            k = rng.integers(0, 2 ** 63, n, dtype=np.uint64).view(np.int64)
        v = np.arange(n, dtype=np.uint32).view(np.int32)
        k1, v1 = torch.as_tensor(k).cuda(), torch.as_tensor(v).cuda()
        k2, v2 = k1.clone(), v1.clone()
        _call("hlc_sort_pairs", k1, v1, bits)
        _call("hlc_sort_pairs_noalloc", k2, v2, bits)
        assert torch.equal(k1, k2), "keys differ on call %d" % call
        assert torch.equal(v1, v2), "values differ on call %d" % call


def test_noalloc_sort_rejects_sizes_beyond_its_capacity():
    torch.cuda.set_device(0)
    k = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    L = hlc.lib()
    rc = L.hlc_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k.numel(), 4, 32,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == hlc.HLC_EINVAL
    assert b"1048576" in L.hlc_last_error()
