"""Batch runtime: many instances sharing the GPU with continuous admission.

Each instance's result in the mix must equal the same instance run alone
(bitwise: every reduction has a fixed order), and match the oracle's picks
where its top-two gap exceeds 1e-6 relative."""
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


def make_specs():
    rng = np.random.default_rng(5)
    specs = []
    for i, (n, d) in enumerate([(500, 16), (3000, 33), (12000, 64), (800, 128), (7000, 16), (2500, 100),
                                 (300, 7), (9000, 128), (1500, 64), (4000, 32)]):
        V = synth.zscore_to_f32(synth.gaussian_mixture(rng, n, d, int(rng.integers(4, 20)), sigma=None))
        prec = ["bf16", "fp16", "fp32"][i % 3] if d <= 128 else "fp32"
        specs.append((V, int(rng.integers(3, 13)), prec))
    return specs


def alone(V, k, prec):
    with ebc.Instance(V, precision=prec) as inst:
        return inst.greedy_host(k)


def test_batch_results_equal_alone(torch):
    specs = make_specs()
    with ebc.Batch(max_slots=4, budget_bytes=8 << 30) as b:
        tickets = [b.submit(V, k, prec) for V, k, prec in specs]
        b.run()
        got = [b.poll(t) for t in tickets]
        st = b.stats()
    assert st["completed"] == len(specs) and st["active"] == 0 and st["queued"] == 0
    for (V, k, prec), res in zip(specs, got):
        assert res is not None
        idx, f = res
        ridx, rf = alone(V, k, prec)
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)


def test_batch_matches_oracle_small(torch):
    specs = make_specs()[:3]
    with ebc.Batch(max_slots=8) as b:
        tickets = [b.submit(V, k, prec) for V, k, prec in specs]
        b.run()
        for (V, k, prec), t in zip(specs, tickets):
            idx, f = b.poll(t)
            ref_idx, ref_f, gap = oracle.greedy(V, k)
            for r in range(k):
                if gap[r] > 1e-6:
                    assert idx[r] == ref_idx[r]
                if idx[r] != ref_idx[r]:
                    break
            np.testing.assert_allclose(f, ref_f, rtol=1e-5)


def test_batch_budget_limits_admission(torch):
    specs = make_specs()[:6]
    est = [ebc.ebc_estimate_bytes(V.shape[0], V.shape[1], ebc.PRECISIONS[p]) for V, _, p in specs]
    budget = sorted(est)[-1] + sorted(est)[-2]  # room for the two largest together at most
    with ebc.Batch(max_slots=6, budget_bytes=budget) as b:
        tickets = [b.submit(V, k, prec) for V, k, prec in specs]
        peak_active = 0
        while True:
            a, q = b.step()
            peak_active = max(peak_active, a)
            if a == 0 and q == 0:
                break
        st = b.stats()
        for t in tickets:
            assert b.poll(t) is not None
    assert st["bytes_peak"] <= budget
    assert st["completed"] == 6


def test_batch_incremental_submission(torch):
    # requests submitted while others are running are admitted without draining
    specs = make_specs()
    with ebc.Batch(max_slots=3) as b:
        first = [b.submit(V, k, p) for V, k, p in specs[:3]]
        b.step()
        b.step()
        later = [b.submit(V, k, p) for V, k, p in specs[3:6]]
        results = {}
        while len(results) < 6:
            b.step()
            for t in first + later:
                if t not in results:
                    r = b.poll(t)
                    if r is not None:
                        results[t] = r
    for (V, k, p), t in zip(specs[:6], first + later):
        ridx, rf = alone(V, k, p)
        np.testing.assert_array_equal(results[t][0], ridx)


def test_batch_errors(torch):
    with ebc.Batch(max_slots=2) as b:
        V = np.zeros((10, 4), np.float32)
        with pytest.raises(ebc.EbcError):
            b.submit(V, 11)
        with pytest.raises(ebc.EbcError):
            b.submit(np.zeros((10, 200), np.float32), 2, "fp8")   # FP8 holds d <= 128
        with pytest.raises(ebc.EbcError):
            b.submit(np.zeros((10, 4097), np.float32), 2, "bf16")  # d <= 4096
        t = b.submit(np.random.default_rng(0).standard_normal((50, 4)).astype(np.float32), 3, "fp32")
        b.run()
        assert b.poll(t) is not None


def test_batch_large_class_limits(torch):
    # instances with n >= 5000 count as large: capped CTAs, one at a time;
    # small ones may start while a large one waits; results as alone
    specs = make_specs()
    with ebc.Batch(max_slots=4) as b:
        b.set_large(5000, 40, 1)
        tickets = [b.submit(V, k, p) for V, k, p in specs]
        b.run()
        res = [b.poll(t) for t in tickets]
    for (V, k, p), r in zip(specs, res):
        ridx, rf = alone(V, k, p)
        np.testing.assert_array_equal(r[0], ridx)
        np.testing.assert_allclose(r[1], rf, rtol=1e-12)
