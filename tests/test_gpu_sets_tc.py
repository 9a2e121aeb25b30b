"""GPU parity of the tensor-core multi-set evaluation (ebc_eval_sets at BF16 /
FP16) against the CPU oracle.

The tensor-core value of a set is raw low-precision arithmetic: each term
max(0, ||v||^2 - min_s dhat(v, s)) uses quantised rows and FP32 tensor-core
accumulation.  Its error is checked against a rigorous bound computed here on
the host from the quantised rows (rounding emulated bit-exactly):
    |fhat_j - f_j| <= (1/n) sum_v max_{s in S_j} E(v, s) + 1e-6 |f_j|
    E(v, s) = (dv + ds)(2 ||v - s|| + dv + ds)                 quantisation
            + gamma (2 ||v_hat|| ||s_hat|| + ||s_hat||^2 + |nv - ||v_hat||^2|)
            + 2^-22 (|nv - ||v_hat||^2| + ||s_hat||^2)          extension split
with dv = ||v_hat - v||, gamma = ((DP + 16)/4 + 4) 2^-22.  The max over s of
a perturbed minimum moves by at most the largest perturbation, and relu is
1-Lipschitz.  The observed error is printed, far below the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import ebc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2105_12026_gb300 import build
    build.build()
    ebc.load()
    t.cuda.set_device(0)
    return t


def quantize_host(V, prec):
    x = np.ascontiguousarray(V, dtype=np.float32)
    if prec == "fp16":
        return x.astype(np.float16).astype(np.float64)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sets_error_bound(V, idx, off, prec, f_ref):
    X = V.astype(np.float64)
    Q = quantize_host(V, prec)
    dq = np.sqrt(((Q - X) ** 2).sum(1))
    qn = (Q ** 2).sum(1)
    qnorm = np.sqrt(qn)
    nv = (X ** 2).sum(1)
    b = np.abs(nv - qn)
    DP = ((V.shape[1] + 63) // 64) * 64
    gamma = ((DP + 16) / 4 + 4) * 2.0 ** -22
    n = V.shape[0]
    out = np.zeros(len(off) - 1)
    for j in range(len(off) - 1):
        mem = idx[off[j]:off[j + 1]]
        if mem.size == 0:
            continue
        S = X[mem]
        dist = np.sqrt(np.maximum(nv[:, None] + nv[mem][None, :] - 2 * X @ S.T, 0))
        dd = dq[:, None] + dq[mem][None, :]
        E = dd * (2 * dist + dd)
        E += gamma * (2 * qnorm[:, None] * qnorm[mem][None, :] + qn[mem][None, :] + b[:, None])
        E += 2.0 ** -22 * (b[:, None] + qn[mem][None, :])
        out[j] = E.max(1).sum() / n
    return out + 1e-6 * np.abs(f_ref) + 1e-12


def run_both(V, idx, off, prec):
    ref = oracle.eval_sets(V, idx, off)
    with ebc.Instance(V, precision=prec) as inst:
        out = inst.eval_sets_host(idx, off)
    return out, ref


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_sets_tc_small_first(torch, prec):
    # one tiny case first: 300 points, 5 sets, one chunk, one point unit
    V = synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(1), 300, 16, 4, sigma=None))
    idx, off = synth.random_sets(np.random.default_rng(2), 300, 5, 1, 20)
    out, ref = run_both(V, idx, off, prec)
    bound = sets_error_bound(V, idx, off, prec, ref)
    err = np.abs(out - ref)
    assert np.isfinite(out).all()
    assert (err <= bound).all(), (err, bound)
    print(prec, "max abs err", err.max(), "max rel", (err / np.maximum(ref, 1e-12)).max(), "bound/err",
          (bound / np.maximum(err, 1e-300)).min())


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,l,smax", [(3000, 64, 200, 64), (777, 33, 90, 40), (4099, 128, 150, 64),
                                        (1000, 1, 30, 8), (2500, 100, 300, 5)])
def test_sets_tc_within_bound(torch, prec, n, d, l, smax):
    rng = np.random.default_rng(n + d + l)
    V = synth.zscore_to_f32(synth.gaussian_mixture(rng, n, d, 8, sigma=None))
    idx, off = synth.random_sets(rng, n, l, 1, min(smax, n))
    out, ref = run_both(V, idx, off, prec)
    bound = sets_error_bound(V, idx, off, prec, ref)
    err = np.abs(out - ref)
    assert (err <= bound).all(), (np.argmax(err - bound), err.max(), bound.min())
    rel = err / np.maximum(ref, 1e-12)
    print(prec, n, d, l, "max rel err", rel.max())


@pytest.mark.parametrize("prec", ["bf16"])
def test_sets_tc_chunking_edge_cases(torch, prec):
    # empty sets (a run of 100 in a row: more than one chunk's worth), a set
    # larger than a chunk, single-member sets, duplicate members, sets that
    # straddle tile and chunk boundaries
    n, d = 2100, 24
    V = synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(5), n, d, 6, sigma=None))
    rng = np.random.default_rng(6)
    sets = [[]] * 100 + [list(rng.choice(n, 2100, replace=False))] + [[7]] * 70 + [[3, 3, 3, 9]]
    sets += [list(rng.choice(n, int(s), replace=True)) for s in rng.integers(1, 300, 40)] + [[]]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    idx = np.concatenate([np.asarray(s, np.int32) for s in sets if len(s)]).astype(np.int32)
    out, ref = run_both(V, idx, off, prec)
    bound = sets_error_bound(V, idx, off, prec, ref)
    assert (out[:100] == 0).all() and out[-1] == 0
    assert (np.abs(out - ref) <= bound).all()


def test_sets_tc_errors_and_determinism(torch):
    V = synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(9), 1500, 40, 5, sigma=None))
    idx, off = synth.random_sets(np.random.default_rng(10), 1500, 64, 1, 64)
    with ebc.Instance(V, precision="bf16") as inst:
        a = inst.eval_sets_host(idx, off)
        b = inst.eval_sets_host(idx, off)
        np.testing.assert_array_equal(a, b)
        # device form, same values
        dev = inst.eval_sets(torch.from_numpy(idx), torch.from_numpy(off)).cpu().numpy()
        np.testing.assert_array_equal(dev, a)
        # out-of-range member: EINDEX at the next sync; the handle stays usable
        bad = idx.copy()
        bad[5] = 1500
        with pytest.raises(ebc.EbcError) as ei:
            inst.eval_sets(torch.from_numpy(bad), torch.from_numpy(off))
            inst.sync()
        assert ei.value.status == ebc.EBC_EINDEX
        # decreasing offsets: EINVAL, found by the device plan and returned by the next sync
        off2 = off.copy()
        off2[3], off2[4] = off2[4], off2[3]
        with pytest.raises(ebc.EbcError) as ei:
            inst.eval_sets(torch.from_numpy(idx), torch.from_numpy(off2))
            inst.sync()
        assert ei.value.status == ebc.EBC_EINVAL
        np.testing.assert_array_equal(inst.eval_sets_host(idx, off), a)
        # the FP32 path on the same handle agrees within the bound
        inst.set_precision("fp32")
        f32 = inst.eval_sets_host(idx, off)
    ref = oracle.eval_sets(V, idx, off)
    assert (np.abs(a - ref) <= sets_error_bound(V, idx, off, "bf16", ref)).all()
    np.testing.assert_allclose(f32, ref, rtol=1e-5, atol=1e-9)


def test_sets_tc_multiset_workload_sampled(torch):
    """n=50,000, d=64, 1,024 sets of size U{1..64}: every set on the GPU, a
    sample of 48 checked against the oracle within the bound."""
    w = synth.multiset_eval(seed=0)
    V, idx, off = w["V"], w["idx"], w["off"]
    with ebc.Instance(V, precision="bf16") as inst:
        out = inst.eval_sets_host(idx, off)
        inst.set_precision("fp32")
        f32 = inst.eval_sets_host(idx, off)
    pick = np.random.default_rng(0).choice(len(off) - 1, 48, replace=False)
    sub_off = np.zeros(49, np.int64)
    sub_off[1:] = np.cumsum(off[pick + 1] - off[pick])
    sub_idx = np.concatenate([idx[off[j]:off[j + 1]] for j in pick]).astype(np.int32)
    ref = oracle.eval_sets(V, sub_idx, sub_off)
    bound = sets_error_bound(V, sub_idx, sub_off, "bf16", ref)
    err = np.abs(out[pick] - ref)
    assert (err <= bound).all()
    np.testing.assert_allclose(f32[pick], ref, rtol=1e-5)
    print("C1 sample: max rel err bf16", (err / ref).max(), "fp32", (np.abs(f32[pick] - ref) / ref).max())


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_sets_tc_device_plan_async_and_capturable(torch, prec):
    """The set plan is made on the device; with a reservation the call reads
    nothing back to the host, so it can be captured in a CUDA graph.  The
    replay gives the same values as the direct call, which equal the
    K-blocked kernel's bitwise (the same MMA sequence), across empty sets,
    sets spanning many tiles and several chunks; a call with more members
    than the reservation holds is rejected on the device."""
    rng = np.random.default_rng(21)
    n, d = 20_000, 48
    V = synth.zscore_to_f32(rng.standard_normal((n, d)))
    sizes = rng.integers(0, 70, size=600)
    sizes[::37] = 0                    # empty sets, some in runs
    sizes[5] = 1500                    # a set spanning six tiles
    sizes[6:9] = 0
    off = np.zeros(sizes.size + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    idx = rng.integers(0, n, size=int(off[-1])).astype(np.int32)
    l = sizes.size
    s = torch.cuda.Stream()
    with ebc.Instance(V, precision=prec, stream=s) as inst:
        inst.reserve_sets(l, int(off[-1]))
        idx_d, off_d = torch.from_numpy(idx).cuda(), torch.from_numpy(off).cuda()
        out = torch.zeros(l, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())  # set-up outside capture
        inst.sync()
        direct = out.cpu().numpy().copy()
        out.zero_()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ebc.ebc_eval_sets(inst.h, idx_d.data_ptr(), off_d.data_ptr(), l, out.data_ptr())
        g.replay()
        s.synchronize()
        inst.sync()
        replay = out.cpu().numpy().copy()
        inst.set_kblocked(True)
        kb = inst.eval_sets_host(idx, off)
        inst.set_kblocked(False)
        # more members than the buffers hold: EINVAL from the device plan
        inst.reserve_sets(2, 16)
        big = torch.from_numpy(np.array([0, 20000, 40000], np.int64)).cuda()
        many = torch.zeros(40000, dtype=torch.int32, device="cuda")
        ebc.ebc_eval_sets(inst.h, many.data_ptr(), big.data_ptr(), 2, out.data_ptr())
        with pytest.raises(ebc.EbcError) as ei:
            inst.sync()
        assert ei.value.status == ebc.EBC_EINVAL
    np.testing.assert_array_equal(replay, direct)
    np.testing.assert_array_equal(direct, kb)
    assert np.all(direct[sizes == 0] == 0.0)
    ref = oracle.eval_sets(V, idx, off)
    bound = sets_error_bound(V, idx, off, prec, ref)
    assert np.all(np.abs(direct - ref) <= bound), np.max(np.abs(direct - ref) - bound)


def test_sets_tc_device_plan_errors(torch):
    V = synth.plain_greedy_small(seed=4)["V"]
    with ebc.Instance(V, precision="bf16") as inst:
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        idx = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
        for bad in ([1, 2, 3], [0, 3, 2]):
            off = torch.tensor(bad, dtype=torch.int64, device="cuda")
            ebc.ebc_eval_sets(inst.h, idx.data_ptr(), off.data_ptr(), 2, out.data_ptr())
            with pytest.raises(ebc.EbcError) as ei:
                inst.sync()
            assert ei.value.status == ebc.EBC_EINVAL
        off = torch.tensor([0, 2, 3], dtype=torch.int64, device="cuda")
        bad_idx = torch.tensor([1, 5000, 3], dtype=torch.int32, device="cuda")
        ebc.ebc_eval_sets(inst.h, bad_idx.data_ptr(), off.data_ptr(), 2, out.data_ptr())
        with pytest.raises(ebc.EbcError) as ei:
            inst.sync()
        assert ei.value.status == ebc.EBC_EINDEX
        # a good call afterwards
        got = inst.eval_sets_host(np.array([1, 2, 3], np.int32), np.array([0, 2, 3], np.int64))
        ref = oracle.eval_sets(V, np.array([1, 2, 3], np.int32), np.array([0, 2, 3], np.int64))
        np.testing.assert_allclose(got, ref, rtol=1e-2)
