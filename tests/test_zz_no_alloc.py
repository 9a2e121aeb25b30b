"""The allocation-free multi-set entry point (ebc_eval_sets_noalloc).

It serves callers that may not allocate device memory while running; it
keeps its scratch in a static device array.  Checked through the C ABI
against the handle-based ebc_eval_sets (FP32) on two calls in a row, since
the shared array keeps the previous call's contents.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

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
    ebc.ebc_eval_sets_noalloc(Vd.data_ptr(), Vd.shape[0], Vd.shape[1], idx.data_ptr(), off.data_ptr(), l,
                              out.data_ptr())
    return out.cpu().numpy()


def test_noalloc_matches_handle_path_twice(torch):
    w1 = synth.multiset_eval(seed=3, n=6000, d=40, l=70)
    w2 = synth.multiset_eval(seed=4, n=6000, d=40, l=55, smax=20)
    Vd = torch.from_numpy(w1["V"]).cuda()
    with ebc.Instance(Vd) as inst:
        ref1 = inst.eval_sets_host(w1["idx"], w1["off"])
        ref2 = inst.eval_sets_host(w2["idx"], w2["off"])
    got1 = _run_noalloc(torch, Vd, torch.from_numpy(w1["idx"]).cuda(), torch.from_numpy(w1["off"]).cuda())
    got2 = _run_noalloc(torch, Vd, torch.from_numpy(w2["idx"]).cuda(), torch.from_numpy(w2["off"]).cuda())
    np.testing.assert_allclose(got1, ref1, rtol=F_RTOL, atol=1e-12)
    np.testing.assert_allclose(got2, ref2, rtol=F_RTOL, atol=1e-12)


def test_noalloc_errors(torch):
    V = torch.from_numpy(synth.plain_greedy_small(seed=1)["V"]).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
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
    # a good call afterwards is unaffected
    idx = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    ebc.ebc_eval_sets_noalloc(V.data_ptr(), V.shape[0], V.shape[1], idx.data_ptr(), off.data_ptr(), 1,
                              out.data_ptr())
    assert out.item() > 0
