"""One persistent bulk launch per Greedy round over an uneven mix of handles
(ebc_group_greedy).

Each handle's picks and f values must be bitwise those of ebc_greedy on the
same handle alone (the shared launch changes only the V chunking of the bulk
bounds, and the pick comes from the exact re-evaluation); a sample of the
mix is checked against the FP64 oracle's Greedy (Sec. 3).  Handles the
shared launch does not serve (FP32, lazy, FP8, d > 128) run on their own
inside the same call.
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


def _mix(count, seed, n_hi=20_000, k_hi=20):
    mix = synth.instance_mix(seed=seed, count=count, n_hi=n_hi, k_hi=k_hi)
    return [(m.make(), int(m.k)) for m in mix]


def _alone(V, k, prec, lazy=False):
    with ebc.Instance(V, precision=prec, lazy=lazy) as inst:
        return inst.greedy_host(k)


def _instances(torch, specs, precs, lazy=None):
    lazy = lazy or [False] * len(specs)
    return [ebc.Instance(V, precision=p, stream=torch.cuda.Stream(), lazy=lz)
            for (V, _), p, lz in zip(specs, precs, lazy)]


def test_group_equals_alone_64(torch):
    specs = _mix(64, seed=3)
    precs = ["bf16" if i % 5 else "fp16" for i in range(len(specs))]
    insts = _instances(torch, specs, precs)
    with ebc.Group(lanes=1) as g:
        got = g.greedy_host(insts, [k for _, k in specs])
        st = g.stats()
    for inst in insts:
        inst.close()
    assert st["launches"] == max(k for _, k in specs)  # one shared launch per round
    for (V, k), p, (idx, f) in zip(specs, precs, got):
        ridx, rf = _alone(V, k, p)
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)
    for i in (0, 17, 40, 63):  # a sample against the oracle
        V, k = specs[i]
        ref_i, ref_f, gap = oracle.greedy(V, k)
        idx, f = got[i]
        for t in range(k):
            if gap[t] > 1e-6:
                assert idx[t] == ref_i[t], (i, t, idx.tolist(), ref_i.tolist())
            if idx[t] != ref_i[t]:
                break
        np.testing.assert_allclose(f, ref_f, rtol=1e-5)


def test_group_mixed_paths_and_continuation(torch):
    """FP32, lazy, FP8 and d > 128 handles run on their own in the same call;
    a second call continues every handle's state."""
    specs = _mix(10, seed=4, n_hi=8000, k_hi=12)
    rng = np.random.default_rng(9)
    wide = synth.zscore_to_f32(rng.standard_normal((3000, 200)))
    specs.append((wide, 6))
    precs = ["bf16", "fp32", "bf16", "fp8", "fp16", "bf16", "bf16", "fp32", "bf16", "fp16", "bf16"]
    lazy = [False, False, True, False, False, False, False, False, False, False, False]
    insts = _instances(torch, specs, precs, lazy)
    k1 = [max(1, k // 2) for _, k in specs]
    k2 = [k - a for (_, k), a in zip(specs, k1)]
    with ebc.Group(lanes=3) as g:
        first = g.greedy_host(insts, k1)
        second = g.greedy_host(insts, k2)
    for inst in insts:
        inst.close()
    for (V, k), p, lz, a, b in zip(specs, precs, lazy, first, second):
        ridx, rf = _alone(V, k, p, lz)
        np.testing.assert_array_equal(np.concatenate([a[0], b[0]]), ridx)
        np.testing.assert_array_equal(np.concatenate([a[1], b[1]]), rf)


def test_group_arguments(torch):
    V = synth.plain_greedy_small(seed=1)["V"]
    with ebc.Instance(V, precision="bf16") as a, ebc.Group() as g:
        with pytest.raises(ebc.EbcError) as ei:
            g.greedy([a, a], [2, 2])  # the same handle twice
        assert ei.value.status == ebc.EBC_EINVAL
        with pytest.raises(ebc.EbcError):
            g.greedy([a], [V.shape[0] + 1])  # more rounds than points
        assert g.greedy([a], [0])[0][0].numel() == 0  # nothing to do
        idx, f = g.greedy_host([a], [3])[0]
        ridx, rf = _alone(V, 3, "bf16")
        np.testing.assert_array_equal(idx, ridx)


def test_group_timeout_reaches_every_handle(torch):
    specs = _mix(6, seed=5, n_hi=6000, k_hi=6)
    insts = _instances(torch, specs, ["bf16"] * len(specs))
    try:
        with ebc.Group() as g:
            ebc.ebc_set_wait_limit_ns(1)
            g.greedy(insts, [2] * len(insts))
            for inst in insts:
                with pytest.raises(ebc.EbcError) as ei:
                    inst.sync()
                assert ei.value.status == ebc.EBC_ETIMEOUT
            ebc.ebc_set_wait_limit_ns(0)
            for inst in insts:
                inst.reset()
            got = g.greedy_host(insts, [k for _, k in specs])
    finally:
        ebc.ebc_set_wait_limit_ns(0)
        for inst in insts:
            inst.close()
    for (V, k), (idx, f) in zip(specs, got):
        ridx, rf = _alone(V, k, "bf16")
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)
