"""The allocation-free multi-set entry point (ebc_eval_sets_noalloc).

It serves callers that may not allocate device memory while running; it
keeps its scratch in a static device array.  Checked through the C ABI
against the handle-based ebc_eval_sets (FP32) on two calls in a row, since
the shared array keeps the previous call's contents, and against the FP64
oracle.  The other cases reach the branches most likely to hide an indexing
mistake: several passes over the array, rows staged in pieces (d > 256), the
grid's 65,535-block limit on set groups, empty sets and offsets that the
device rejects.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import ebc, synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2105_12026_gb300 import build
    build.build()
    ebc.load()
    t.cuda.set_device(0)
    return t


def _run_noalloc(torch, Vd, idx, off):
    l = off.numel() - 1
    out = torch.full((l,), -1.0, dtype=torch.float64, device="cuda")
    ebc.ebc_eval_sets_noalloc(Vd.data_ptr(), Vd.shape[0], Vd.shape[1], idx.data_ptr() if idx is not None else 0,
                              off.data_ptr(), l, out.data_ptr())
    return out.cpu().numpy()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_handle_path_twice(torch):
    w1 = synth.multiset_eval(seed=3, n=6000, d=40, l=70)
    w2 = synth.multiset_eval(seed=4, n=6000, d=40, l=55, smax=20)
    Vd = torch.from_numpy(w1["V"]).cuda()
    with ebc.Instance(Vd) as inst:
        ref1 = inst.eval_sets_host(w1["idx"], w1["off"])
        ref2 = inst.eval_sets_host(w2["idx"], w2["off"])
    got1 = _run_noalloc(torch, Vd, _dev(torch, w1["idx"]), _dev(torch, w1["off"]))
    got2 = _run_noalloc(torch, Vd, _dev(torch, w2["idx"]), _dev(torch, w2["off"]))
    np.testing.assert_allclose(got1, ref1, rtol=F_RTOL, atol=1e-12)
    np.testing.assert_allclose(got2, ref2, rtol=F_RTOL, atol=1e-12)
    # and against the FP64 definition
    np.testing.assert_allclose(got1, oracle.eval_sets(w1["V"], w1["idx"], w1["off"]), rtol=F_RTOL, atol=1e-12)
    np.testing.assert_allclose(got2, oracle.eval_sets(w1["V"], w2["idx"], w2["off"]), rtol=F_RTOL, atol=1e-12)


def test_noalloc_several_passes(torch):
    # 2,344 tiles of 128 points: 447 sets fit the array per pass, 500 take two
    rng = np.random.default_rng(11)
    V = synth.zscore_to_f32(rng.standard_normal((300_000, 16)))
    idx, off = synth.random_sets(rng, V.shape[0], 500, 1, 8)
    Vd = _dev(torch, V)
    got = _run_noalloc(torch, Vd, _dev(torch, idx), _dev(torch, off))
    with ebc.Instance(Vd) as inst:
        ref = inst.eval_sets_host(idx, off)
    np.testing.assert_allclose(got, ref, rtol=F_RTOL, atol=1e-12)
    pick = np.sort(rng.choice(500, 24, replace=False))
    sub_off = np.concatenate([[0], np.cumsum(off[pick + 1] - off[pick])]).astype(np.int64)
    sub_idx = np.concatenate([idx[off[j]:off[j + 1]] for j in pick]).astype(np.int32)
    np.testing.assert_allclose(got[pick], oracle.eval_sets(V, sub_idx, sub_off), rtol=F_RTOL, atol=1e-12)


def test_noalloc_many_small_sets_grid_limit(torch):
    # n = 200 (two tiles): the array would hold 524,288 sets per pass, more set
    # groups than a grid's y extent allows; 600,000 one-member sets need two passes
    rng = np.random.default_rng(12)
    V = synth.zscore_to_f32(rng.standard_normal((200, 8)))
    l = 600_000
    idx = rng.integers(0, V.shape[0], size=l).astype(np.int32)
    off = np.arange(l + 1, dtype=np.int64)
    Vd = _dev(torch, V)
    got = _run_noalloc(torch, Vd, _dev(torch, idx), _dev(torch, off))
    ref = oracle.eval_sets(V, idx, off)
    np.testing.assert_allclose(got, ref, rtol=F_RTOL, atol=1e-12)
    # the handle path at FP32 has the same limit on its set groups
    with ebc.Instance(Vd) as inst:
        got_h = inst.eval_sets(_dev(torch, idx), _dev(torch, off)).cpu().numpy()
    np.testing.assert_allclose(got_h, ref, rtol=F_RTOL, atol=1e-12)


def test_noalloc_rows_staged_in_pieces(torch):
    # d = 300 > 256: every member row is staged in two pieces
    rng = np.random.default_rng(13)
    V = synth.zscore_to_f32(rng.standard_normal((2000, 300)))
    idx, off = synth.random_sets(rng, V.shape[0], 40, 1, 12)
    got = _run_noalloc(torch, _dev(torch, V), _dev(torch, idx), _dev(torch, off))
    np.testing.assert_allclose(got, oracle.eval_sets(V, idx, off), rtol=F_RTOL, atol=1e-12)


def test_noalloc_empty_sets(torch):
    V = synth.plain_greedy_small(seed=2)["V"]
    Vd = _dev(torch, V)
    idx = np.array([3, 7, 7, 100], dtype=np.int32)
    off = np.array([0, 0, 2, 2, 4, 4], dtype=np.int64)  # sets: {}, {3,7}, {}, {7,100}, {}
    got = _run_noalloc(torch, Vd, _dev(torch, idx), _dev(torch, off))
    ref = oracle.eval_sets(V, idx, off)
    assert got[0] == 0.0 and got[2] == 0.0 and got[4] == 0.0
    np.testing.assert_allclose(got, ref, rtol=F_RTOL, atol=1e-12)
    # only empty sets: a NULL member list is allowed and gives zeros
    off0 = np.zeros(4, dtype=np.int64)
    got0 = _run_noalloc(torch, Vd, None, _dev(torch, off0))
    assert got0.tolist() == [0.0, 0.0, 0.0]


def test_noalloc_errors(torch):
    V = torch.from_numpy(synth.plain_greedy_small(seed=1)["V"]).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad_idx = torch.tensor([1, 5000], dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 2], dtype=torch.int64, device="cuda")
    with pytest.raises(ebc.EbcError) as ei:
        ebc.ebc_eval_sets_noalloc(V.data_ptr(), V.shape[0], V.shape[1], bad_idx.data_ptr(), off.data_ptr(), 1,
                                  out.data_ptr())
    assert ei.value.status == ebc.EBC_EINDEX
    with pytest.raises(ebc.EbcError) as ei:
        ebc.ebc_eval_sets_noalloc(V.data_ptr(), 1 << 28, V.shape[1], bad_idx.data_ptr(), off.data_ptr(), 1,
                                  out.data_ptr())
    assert ei.value.status == ebc.EBC_EINVAL and "scratch" in str(ei.value)
    idx = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
    # offsets that do not start at 0, and offsets that decrease, are found on the device
    for bad_off in ([1, 2, 3], [0, 3, 2]):
        o = torch.tensor(bad_off, dtype=torch.int64, device="cuda")
        with pytest.raises(ebc.EbcError) as ei:
            ebc.ebc_eval_sets_noalloc(V.data_ptr(), V.shape[0], V.shape[1], idx.data_ptr(), o.data_ptr(), 2,
                                      out.data_ptr())
        assert ei.value.status == ebc.EBC_EINVAL
    # a good call afterwards is unaffected
    idx2 = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    ebc.ebc_eval_sets_noalloc(V.data_ptr(), V.shape[0], V.shape[1], idx2.data_ptr(), off.data_ptr(), 1,
                              out.data_ptr())
    ref = oracle.eval_sets(V.cpu().numpy(), np.array([1, 2], np.int32), np.array([0, 2], np.int64))
    np.testing.assert_allclose(out[:1].cpu().numpy(), ref, rtol=F_RTOL)
