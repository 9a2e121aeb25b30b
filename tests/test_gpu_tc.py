"""GPU parity of the tensor-core (tcgen05) precisions against the CPU oracle.

* Greedy with BF16 / FP16 bulk gains: the picks are certified by exact FP64
  re-evaluation, so they must equal the oracle's wherever its top-two gap
  exceeds 1e-6 relative, and f must agree within 1e-5 relative.
* ebc_gains at a tensor-core precision returns the raw low-precision gain;
  its error is checked against a rigorous bound computed here on the host
  from the quantised rows (rounding emulated bit-exactly in numpy):
      |g_raw - g| <= max_c [Dl (2 sqrt(M) + Dl) + 2 gamma |v|max |c|] + eps
  with Dl = max|v_hat - v| + |c_hat - c|, M = max m_v.  The observed error is
  reported, far below the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import ebc, synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-5
PICK_GAP = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2105_12026_gb300 import build
    build.build()
    ebc.load()
    t.cuda.set_device(0)
    return t


def quantize_host(V, prec):
    """Round-to-nearest-even FP32 -> bf16 / fp16, returned as FP64."""
    x = np.ascontiguousarray(V, dtype=np.float32)
    if prec == "fp16":
        return x.astype(np.float16).astype(np.float64)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def raw_error_bound(V, m, prec):
    Vq = quantize_host(V, prec)
    err = np.sqrt(((Vq - V.astype(np.float64)) ** 2).sum(1))
    qn = np.sqrt((Vq ** 2).sum(1))
    M = float(m.max())
    dl = err.max() + err
    K = ((V.shape[1] + 63) // 64) * 64
    gamma = K * 2.0 ** -20
    Ec = dl * (2 * np.sqrt(M) + dl) + 2 * gamma * qn.max() * qn
    Z = 2 * qn.max() * qn + qn.max() ** 2 + M + qn ** 2
    return Ec + Z * 2.0 ** -21


def check_greedy(idx, f, ref_idx, ref_f, ref_gap):
    diverged = False
    for t in range(len(ref_idx)):
        if not diverged and ref_gap[t] > PICK_GAP:
            assert idx[t] == ref_idx[t], f"round {t}: gpu {idx[t]} oracle {ref_idx[t]} gap {ref_gap[t]}"
        if idx[t] != ref_idx[t]:
            diverged = True
    np.testing.assert_allclose(f, ref_f, rtol=F_RTOL)
    return diverged


def gmm(n, d, seed, clusters=6):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, clusters, sigma=None))


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_gains_small_first(torch, prec):
    # one small case first: 300 points, d = 16, a single tile in each direction
    V = gmm(300, 16, 1)
    ref = oracle.gains(V, oracle.norms(V), np.arange(300, dtype=np.int32))
    with ebc.Instance(V, precision=prec) as inst:
        g = inst.gains_host(None)
    bound = raw_error_bound(V, oracle.norms(V), prec)
    err = np.abs(g - ref)
    assert np.isfinite(g).all()
    assert (err <= bound + 1e-9).all(), (err.max(), bound.min())
    print(prec, "raw max abs err", err.max(), "rel", (err / np.maximum(ref, 1e-12)).max())


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d", [(1, 1), (129, 3), (257, 64), (1000, 100), (4099, 128), (700, 33)])
def test_tc_gains_raw_within_bound(torch, prec, n, d):
    V = gmm(n, d, n + d) if n > 8 else np.random.default_rng(0).standard_normal((n, d)).astype(np.float32)
    m = oracle.norms(V)
    ref = oracle.gains(V, m, np.arange(n, dtype=np.int32))
    with ebc.Instance(V, precision=prec) as inst:
        g = inst.gains_host(None)
        cand = np.arange(n, dtype=np.int32)[::-1].copy()
        g2 = inst.gains_host(cand)
    bound = raw_error_bound(V, m, prec)
    assert (np.abs(g - ref) <= bound + 1e-9).all()
    np.testing.assert_array_equal(g2, g[::-1])


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tc_greedy_plain_small_workload(torch, prec):
    w = synth.plain_greedy_small(seed=0)
    V, k = w["V"], w["k"]
    ref = oracle.greedy(V, k)
    with ebc.Instance(torch.from_numpy(V).cuda(), precision=prec) as inst:
        idx, f = inst.greedy_host(k)
        st = inst.stats()
    assert not check_greedy(idx, f, *ref)
    assert idx.tolist() == ref[0].tolist()
    np.testing.assert_allclose(f, ref[1], rtol=1e-12)
    assert st["certified_rounds"] + st["escalated_rounds"] == k
    print(prec, st)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,k", [(1, 1, 1), (2, 5, 2), (300, 17, 8), (2000, 64, 12), (5000, 128, 10),
                                   (777, 100, 20)])
def test_tc_greedy_ragged(torch, prec, n, d, k):
    V = gmm(n, d, 3 * n + d) if n > 8 else np.random.default_rng(n).standard_normal((n, d)).astype(np.float32)
    ref = oracle.greedy(V, k)
    with ebc.Instance(V, precision=prec) as inst:
        idx, f = inst.greedy_host(k)
    check_greedy(idx, f, *ref)


def test_tc_greedy_duplicates_to_exhaustion(torch):
    base = gmm(40, 8, 5)
    V = np.concatenate([base, base[:13], base[7:9]], 0)
    n = V.shape[0]
    ref = oracle.greedy(V, n)
    with ebc.Instance(V, precision="bf16") as inst:
        idx, f = inst.greedy_host(n)
        st = inst.stats()
    assert sorted(idx.tolist()) == list(range(n))
    check_greedy(idx, f, *ref)
    assert st["exact_evaluations"] >= n  # at least one contender per round


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
def test_refine_k1_forces_escalation(torch, prec):
    # with a single leader the (K+1)-th bulk bound nearly always reaches the
    # leader's lower bound, so the escalation path decides most rounds
    V = gmm(3000, 24, 77, clusters=5)
    ref = oracle.greedy(V, 12)
    with ebc.Instance(V, precision=prec, refine_k=1) as inst:
        idx, f = inst.greedy_host(12)
        st = inst.stats()
    check_greedy(idx, f, *ref)
    assert st["escalated_rounds"] > 0
    assert st["certified_rounds"] + st["escalated_rounds"] == 12


def test_tc_switch_precision_and_reload(torch):
    V1 = gmm(3000, 48, 11)
    V2 = gmm(3000, 48, 12)
    r1 = oracle.greedy(V1, 6)
    r2 = oracle.greedy(V2, 6)
    with ebc.Instance(torch.from_numpy(V1).cuda()) as inst:
        i32, f32 = inst.greedy_host(6)
        inst.reset()
        inst.set_precision("bf16")
        ib, fb = inst.greedy_host(6)
        inst.reload(torch.from_numpy(V2).cuda())  # re-quantises
        i2, f2 = inst.greedy_host(6)
        inst.set_precision("fp16")
        inst.reset()
        ih, fh = inst.greedy_host(6)
    check_greedy(i32, f32, *r1)
    check_greedy(ib, fb, *r1)
    check_greedy(i2, f2, *r2)
    check_greedy(ih, fh, *r2)


def test_tc_rejects_fp16_overflow_and_fp8_large_d(torch):
    V = gmm(100, 8, 1)
    V[3, 2] = 1e6
    with ebc.Instance(V) as inst:
        with pytest.raises(ebc.EbcError) as ei:
            inst.set_precision("fp16")
        assert ei.value.status == ebc.EBC_EINVAL
        inst.set_precision("bf16")  # bf16 has the range
        inst.greedy_host(2)
    W = gmm(50, 200, 2)
    with ebc.Instance(W) as inst:
        inst.set_precision("bf16")  # d > 128: the K-blocked kernel
        with pytest.raises(ebc.EbcError) as ei:
            inst.set_precision("fp8")
        assert ei.value.status == ebc.EBC_EINVAL


def test_tc_deterministic(torch):
    V = gmm(20000, 128, 4)
    with ebc.Instance(V, precision="bf16") as a, ebc.Instance(V, precision="bf16") as b:
        ia, fa = a.greedy_host(5)
        ib, fb = b.greedy_host(5)
        ga, gb = a.gains_host(None), b.gains_host(None)
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(ga, gb)
