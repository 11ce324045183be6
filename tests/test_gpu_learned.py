"""GPU parity of the learned offset index: every lookup (present keys, absent
keys, keys outside the range) equals the plain binary-search lower bound, for
the piecewise-linear and the MLP models, on uniform and strongly clustered
key sets; and whole matches through the learned index equal the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2301_07331_b300 as hlc
from paper_2301_07331_b300 import synth

pytestmark = pytest.mark.gpu


def _keys(kind, n, bits, rng):
    if kind == "uniform":
        k = rng.integers(0, 2 ** bits, n, dtype=np.uint64)
    else:  # clustered: a few dense clumps plus a sparse background
        centres = rng.integers(0, 2 ** bits, 20, dtype=np.uint64)
        k = np.concatenate([
            (centres[rng.integers(0, 20, n * 9 // 10)].astype(np.int64)
             + rng.normal(0, 2 ** (bits - 14), n * 9 // 10).astype(np.int64)).clip(0, 2 ** bits - 1).astype(np.uint64),
            rng.integers(0, 2 ** bits, n - n * 9 // 10, dtype=np.uint64)])
    return np.unique(k).astype(np.uint32)


@pytest.mark.parametrize("model", [hlc.HLC_MODEL_PLA, hlc.HLC_MODEL_MLP, hlc.HLC_MODEL_NONE])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
@pytest.mark.parametrize("bits,shift", [(28, 20), (30, 24), (32, 24), (20, 8), (12, 0)])
def test_lookup_equals_binary_search(model, kind, bits, shift):
    rng = np.random.default_rng(bits + shift)
    uniq = _keys(kind, 200_000, bits, rng)
    q = np.concatenate([uniq[rng.integers(0, uniq.size, 50_000)],          # present
                        rng.integers(0, 2 ** bits, 50_000, dtype=np.uint64).astype(np.uint32),
                        np.array([0, 2 ** bits - 1, uniq[0], uniq[-1], uniq[-1] + 1], dtype=np.uint32),
                        np.array([2 ** 32 - 1], dtype=np.uint32)])
    tu = torch.as_tensor(uniq.view(np.int32)).cuda()
    tq = torch.as_tensor(q.view(np.int32)).cuda()
    got, st = hlc.hlc_learned_lookup(tu, shift, model, tq)
    want = np.searchsorted(uniq, q, side="left")
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want)
    assert st["learned_models"] >= 1
    if model == hlc.HLC_MODEL_PLA:
        assert st["learned_hit_rate"] == 1.0  # monotone model: always inside the window


def test_lookup_empty_and_tiny():
    for uniq in [np.array([], np.uint32), np.array([7], np.uint32), np.array([0, 5, 9], np.uint32)]:
        q = np.array([0, 1, 5, 6, 9, 10, 2 ** 32 - 1], dtype=np.uint32)
        tu = torch.as_tensor(uniq.view(np.int32)).cuda()
        tq = torch.as_tensor(q.view(np.int32)).cuda()
        got, _ = hlc.hlc_learned_lookup(tu, 2, hlc.HLC_MODEL_PLA, tq)
        np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32),
                                      np.searchsorted(uniq, q, side="left"))


@pytest.mark.parametrize("model", [hlc.HLC_MODEL_PLA, hlc.HLC_MODEL_MLP])
@pytest.mark.parametrize("mode,prec", [(hlc.HLC_COMPLETE8, hlc.HLC_FP32_GUARD),
                                       (hlc.HLC_COMPLETE8, hlc.HLC_FP64),
                                       (hlc.HLC_QUAD, hlc.HLC_FP32_GUARD)])
def test_match_through_learned_index(model, mode, prec):
    A, B = synth.fullsky_pair(na=200_000, nb=200_000)
    want = O.match(*A.numpy(), *B.numpy(), 1.0, 14, mode)
    dev = lambda X: (X.ra.cuda(), X.dec.cuda(), X.id.cuda())
    plan = hlc.hlc_plan(dev(A), dev(B), 1.0, 14, coarse_level=4, boundary=mode, precision=prec,
                        index=hlc.HLC_INDEX_LEARNED, model=model)
    res = hlc.hlc_match(plan)
    hlc.hlc_free(plan)
    np.testing.assert_array_equal(res["id_a"].cpu().numpy().view(np.uint64), want["id_a"])
    np.testing.assert_array_equal(res["id_b"].cpu().numpy().view(np.uint64), want["id_b"])
    assert np.max(np.abs(res["sep"].cpu().numpy() - want["sep"])) <= 1e-6
    st = res["stats"]
    assert st["learned_models"] == 12 * 4 ** 4
    if model == hlc.HLC_MODEL_PLA:
        assert st["learned_hit_rate"] == 1.0
