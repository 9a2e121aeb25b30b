"""The K-blocked tensor-core bulk kernel (k_gains_tc_kb): candidate and
point rows streamed in 64-element K blocks, for d > 128 at BF16 / FP16.

It issues the same MMA sequence as the resident-row kernel, so where both
apply (d <= 128) the bulk bounds, picks and f must be bitwise the same;
above d = 128 Greedy, lazy Greedy and the threshold sieve must match the
FP64 oracle at the usual bars (picks while the oracle's top-two gap exceeds
1e-6, f within F_RTOL), up to the case-study shape of the paper's Fig. 4
(n = 1,000, d = 3,524).
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


def gmm(n, d, seed, clusters=6):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, clusters, sigma=None))


def check_oracle(idx, f, ref_idx, ref_f, ref_gap):
    diverged = False
    for t in range(len(ref_idx)):
        if not diverged and ref_gap[t] > PICK_GAP:
            assert idx[t] == ref_idx[t], f"round {t}: gpu {idx[t]} oracle {ref_idx[t]} gap {ref_gap[t]}"
        if idx[t] != ref_idx[t]:
            diverged = True
    np.testing.assert_allclose(f, ref_f, rtol=F_RTOL)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,k", [(700, 17, 9), (3000, 64, 12), (5000, 128, 10), (300, 1, 5)])
def test_kblocked_equals_resident_bitwise(torch, prec, n, d, k):
    V = gmm(n, d, n + 3 * d)
    cand = np.random.default_rng(d).choice(n, size=min(n, 777), replace=False).astype(np.int32)
    res = {}
    for kb in (False, True):
        with ebc.Instance(V, precision=prec) as inst:
            inst.set_kblocked(kb)
            g0 = inst.gains_host(cand)
            idx, f = inst.greedy_host(k)
            g1 = inst.gains_host(None)
            inst.reset()
            inst.set_lazy(True)
            li, lf = inst.greedy_host(k)
            res[kb] = (g0, idx, f, g1, li, lf)
    for a, b in zip(res[False], res[True]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,k", [(2000, 129, 10), (1500, 256, 8), (1200, 300, 8), (900, 777, 6),
                                   (640, 2048, 5), (333, 4096, 4)])
def test_large_d_greedy_matches_oracle(torch, prec, n, d, k):
    V = gmm(n, d, 11 * n + d)
    ref = oracle.greedy(V, k)
    with ebc.Instance(V, precision=prec) as inst:
        idx, f = inst.greedy_host(k)
        inst.reset()
        inst.set_lazy(True)
        li, lf = inst.greedy_host(k)
    check_oracle(idx, f, *ref)
    np.testing.assert_array_equal(li, idx)
    np.testing.assert_array_equal(lf, f)


def test_case_study_shape(torch):
    """n = 1,000 time series of d = 3,524 (the shape of the case study,
    Sec. 6, Fig. 4), BF16 Greedy k = 20 against the oracle."""
    rng = np.random.default_rng(5)
    t = np.linspace(0, 1, 3524)
    base = np.stack([np.sin(2 * np.pi * (3 + j) * t) for j in range(8)])
    w = rng.standard_normal((1000, 8))
    X = w @ base + 0.3 * rng.standard_normal((1000, 3524))
    V = synth.zscore_to_f32(X)
    ref = oracle.greedy(V, 20)
    with ebc.Instance(V, precision="bf16") as inst:
        idx, f = inst.greedy_host(20)
    check_oracle(idx, f, *ref)


def test_large_d_sieve_and_gains(torch):
    n, d, K = 1500, 600, 12
    V = gmm(n, d, 77)
    stream = np.random.default_rng(3).permutation(n).astype(np.int32)
    m1 = float(oracle.greedy(V, 1)[1][0])
    ref = oracle.three_sieves(V, stream, K, 0.1, 20, m1)
    with ebc.Instance(V, precision="bf16") as inst:
        idx, f, sv = ebc.three_sieves(inst, stream, K, 0.1, 20, m1)
        inst.reset()
        g = inst.gains_host(np.arange(0, n, 7, dtype=np.int32))
    if np.all(ref["margin"][~np.isnan(ref["margin"])] > 1e-6):
        assert idx.tolist() == ref["idx"].tolist()
        np.testing.assert_allclose(f, ref["f"], rtol=1e-7)
    # raw BF16 gains at S = {}: finite, and their leader is a near-leader exactly
    exact = oracle.gains(V, oracle.norms(V), np.arange(0, n, 7))
    assert np.all(np.isfinite(g)) and np.all(g >= 0)
    assert exact[np.argmax(g)] >= 0.99 * exact.max()


def test_large_d_batch(torch):
    specs = [(gmm(800, 300, 1), 6), (gmm(500, 1000, 2), 4)]
    with ebc.Batch(max_slots=2, budget_bytes=8 << 30) as b:
        tickets = [b.submit(V, k, "bf16") for V, k in specs]
        b.run()
        got = [b.poll(t) for t in tickets]
    for (V, k), (idx, f) in zip(specs, got):
        with ebc.Instance(V, precision="bf16") as inst:
            ridx, rf = inst.greedy_host(k)
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,l", [(3000, 16, 60), (2000, 64, 200), (1500, 128, 90)])
def test_kblocked_sets_equal_resident_bitwise(torch, prec, n, d, l):
    V = gmm(n, d, 5 * n + d)
    idx, off = synth.random_sets(np.random.default_rng(d), n, l, 0, 70)
    got = {}
    for kb in (False, True):
        with ebc.Instance(V, precision=prec) as inst:
            inst.set_kblocked(kb)
            got[kb] = inst.eval_sets_host(idx, off)
    np.testing.assert_array_equal(got[False], got[True])


@pytest.mark.parametrize("n,d,l", [(1200, 200, 80), (900, 777, 50), (1000, 3524, 40)])
def test_large_d_sets_within_bound(torch, n, d, l):
    from test_gpu_sets_tc import sets_error_bound
    V = gmm(n, d, 3 * n + d)
    idx, off = synth.random_sets(np.random.default_rng(n), n, l, 1, 40)
    ref = oracle.eval_sets(V, idx, off)
    with ebc.Instance(V, precision="bf16") as inst:
        got = inst.eval_sets_host(idx, off)
    bound = sets_error_bound(V, idx, off, "bf16", ref)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (np.max(err - bound), d)
    print(d, "max err", err.max(), "max bound", bound.max())
