"""FP8 e4m3 on the tensor cores.

* ebc_gains at EBC_FP8E4M3 returns raw FP8 gains; their error is checked
  against a rigorous bound computed on the host from the quantised rows
  (e4m3 rounding emulated with torch's float8_e4m3fn, round to nearest):
      |g_raw - g| <= max_c [Dl (2 sqrt(M) + Dl) + gamma8 Z_c] + eps,
  Dl = max_v ||v_hat - v|| + ||c_hat - c||, M = max m_v, Z_c the absolute
  sum of the accumulated terms, gamma8 the tensor-core accumulation bound
  the kernel assumes (2^-8 + the FP32 part).
* ebc_greedy at EBC_FP8E4M3 bounds every candidate with FP8, then certifies
  with BF16 bounds: picks and f must be bitwise those of the BF16 Greedy
  (the same exact argmax and exact gain), hence match the oracle too.
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


def gmm(n, d, seed, clusters=6):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, clusters, sigma=None))


def pow2_scale(a):
    a = np.asarray(a, np.float64)
    out = np.ones_like(a)
    pos = a > 0
    out[pos] = 2.0 ** np.ceil(np.log2(a[pos] / 448.0))
    return out


def quantize_fp8(V, torch):
    X = np.asarray(V, np.float32)
    sc = pow2_scale(np.abs(X).max(1))
    t = float(pow2_scale(np.abs(X).max()))
    e4 = lambda A: torch.from_numpy(np.ascontiguousarray(A, np.float32)).to(torch.float8_e4m3fn).double().numpy()
    C = e4(X / sc[:, None]) * sc[:, None]
    P = e4(X / t) * t
    return C, P


def raw_bound(V, m, torch):
    X = V.astype(np.float64)
    C, P = quantize_fp8(V, torch)
    dc = np.sqrt(((C - X) ** 2).sum(1))
    dv = np.sqrt(((P - X) ** 2).sum(1))
    M = float(m.max())
    dl = dv.max() + dc
    K = ((V.shape[1] + 127) // 128) * 128 + 16
    gamma8 = 2.0 ** -8 + (K / 4 + 4) * 2.0 ** -22
    qc, qp = np.sqrt((C ** 2).sum(1)), np.sqrt((P ** 2).sum(1))
    Z = 2 * qp.max() * qc + qc ** 2 + M + qp.max() ** 2
    return dl * (2 * np.sqrt(M) + dl) + gamma8 * Z + 1e-9


def test_fp8_gains_small_first(torch):
    V = gmm(300, 16, 1)
    m = oracle.norms(V)
    ref = oracle.gains(V, m, np.arange(300, dtype=np.int32))
    with ebc.Instance(V, precision="fp8") as inst:
        g = inst.gains_host(None)
    err = np.abs(g - ref)
    assert np.isfinite(g).all()
    assert (err <= raw_bound(V, m, torch)).all()
    print("fp8 raw max abs err", err.max(), "max rel", (err / np.maximum(ref, 1e-12)).max())


@pytest.mark.parametrize("n,d", [(1, 1), (129, 3), (1000, 100), (4099, 128), (700, 33)])
def test_fp8_gains_within_bound_and_lists(torch, n, d):
    V = gmm(n, d, n + d) if n > 8 else np.random.default_rng(0).standard_normal((n, d)).astype(np.float32)
    m = oracle.norms(V)
    ref = oracle.gains(V, m, np.arange(n, dtype=np.int32))
    with ebc.Instance(V, precision="fp8") as inst:
        g = inst.gains_host(None)
        g2 = inst.gains_host(np.arange(n, dtype=np.int32)[::-1].copy())
    assert (np.abs(g - ref) <= raw_bound(V, m, torch)).all()
    np.testing.assert_array_equal(g2, g[::-1])


@pytest.mark.parametrize("n,d,k", [(1, 1, 1), (300, 17, 8), (2000, 64, 12), (5000, 128, 10), (777, 100, 20)])
def test_fp8_greedy_equals_bf16(torch, n, d, k):
    V = gmm(n, d, 3 * n + d) if n > 8 else np.random.default_rng(n).standard_normal((n, d)).astype(np.float32)
    with ebc.Instance(V, precision="bf16") as a:
        ia, fa = a.greedy_host(k)
    with ebc.Instance(V, precision="fp8") as b:
        ib, fb = b.greedy_host(k)
        st = b.stats()
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)
    ref_idx, ref_f, ref_gap = oracle.greedy(V, k)
    np.testing.assert_allclose(fb, ref_f, rtol=1e-5)
    print("fp8", n, d, k, "BF16 second-level candidates", st["bulk_candidates"], "of", sum(n - t for t in range(k)))


def test_fp8_switch_reload_and_batch(torch):
    V1, V2 = gmm(3000, 48, 11), gmm(3000, 48, 12)
    with ebc.Instance(V1, precision="bf16") as ref:
        r1 = ref.greedy_host(6)
        ref.reload(V2)
        r2 = ref.greedy_host(6)
    with ebc.Instance(V1) as inst:
        inst.set_precision("fp8")
        a = inst.greedy_host(6)
        inst.reload(V2)  # re-quantises both copies
        b = inst.greedy_host(6)
        inst.set_precision("fp16")
        inst.reset()
        c = inst.greedy_host(6)
    np.testing.assert_array_equal(a[0], r1[0])
    np.testing.assert_array_equal(b[0], r2[0])
    np.testing.assert_array_equal(c[0], r2[0])
    with ebc.Batch(max_slots=2) as bt:
        t1 = bt.submit(V1, 6, "fp8")
        bt.run()
        got = bt.poll(t1)
    np.testing.assert_array_equal(got[0], r1[0])
    np.testing.assert_array_equal(got[1], r1[1])
