"""Lazy Greedy (ebc_set_lazy) on the GPU.

A lazy round bounds only the candidates whose stale upper bound (from an
earlier round; valid by diminishing returns) reaches a certified lower bound
of the round's best gain, and certifies the pick among them.  Its picks and
f values must be bitwise those of the full round (same exact argmax, same tie
rule, same exact gain kernel), hence also match the oracle at the usual bars;
and it must evaluate fewer candidates once the bounds have warmed up.
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


def full_and_lazy(V, k, prec, refine_k=8, stream=None):
    with ebc.Instance(V, precision=prec, refine_k=refine_k, stream=stream) as a:
        ia, fa = a.greedy_host(k)
    with ebc.Instance(V, precision=prec, refine_k=refine_k, stream=stream, lazy=True) as b:
        ib, fb = b.greedy_host(k)
        st = b.stats()
    return (ia, fa), (ib, fb), st


def test_lazy_small_first(torch):
    w = synth.plain_greedy_small(seed=0)
    V, k = w["V"], w["k"]
    (ia, fa), (ib, fb), st = full_and_lazy(V, k, "bf16")
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)
    check_oracle(ib, fb, *oracle.greedy(V, k))
    assert st["lazy"] == 1 and st["rounds"] == k
    print("bulk candidates", st["bulk_candidates"], "of", sum(V.shape[0] - t for t in range(k)))


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,d,k", [(1, 1, 1), (2, 5, 2), (300, 17, 8), (2000, 64, 12), (5000, 128, 10),
                                   (777, 100, 20), (20000, 32, 40)])
def test_lazy_equals_full(torch, prec, n, d, k):
    V = gmm(n, d, 3 * n + d) if n > 8 else np.random.default_rng(n).standard_normal((n, d)).astype(np.float32)
    (ia, fa), (ib, fb), st = full_and_lazy(V, k, prec)
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)
    full = sum(n - t for t in range(k))
    assert 0 < st["bulk_candidates"] <= full
    if n >= 2000:
        check_oracle(ib, fb, *oracle.greedy(V, k))
        assert st["bulk_candidates"] < 0.6 * full, (st["bulk_candidates"], full)
    print(prec, n, d, k, "bulk candidates", st["bulk_candidates"], "of", full)


def test_lazy_duplicates_to_exhaustion(torch):
    base = gmm(40, 8, 5)
    V = np.concatenate([base, base[:13], base[7:9]], 0)
    n = V.shape[0]
    (ia, fa), (ib, fb), st = full_and_lazy(V, n, "bf16")
    assert sorted(ib.tolist()) == list(range(n))
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_lazy_refine_k1_and_graphs(torch, prec):
    V = gmm(6000, 24, 77, clusters=5)
    s = torch.cuda.Stream()
    (ia, fa), (ib, fb), st = full_and_lazy(V, 15, prec, refine_k=1, stream=s)
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)
    # one-round calls on a stream replay the captured lazy round
    with ebc.Instance(V, precision=prec, refine_k=1, stream=s, lazy=True) as c:
        parts = [c.greedy_host(1) for _ in range(15)]
    np.testing.assert_array_equal(np.concatenate([p[0] for p in parts]), ia)
    np.testing.assert_array_equal(np.concatenate([p[1] for p in parts]), fa)


def test_lazy_toggle_reset_reload(torch):
    V1 = gmm(8000, 40, 11)
    V2 = gmm(8000, 40, 12)
    with ebc.Instance(V1, precision="bf16") as ref:
        r1 = ref.greedy_host(12)
        ref.reload(V2)
        r2 = ref.greedy_host(12)
    with ebc.Instance(V1, precision="bf16") as inst:
        a, fa = inst.greedy_host(5)      # full rounds
        inst.set_lazy(True)              # bounds restart from the current state
        b, fb = inst.greedy_host(4)
        inst.set_lazy(False)
        c, fc = inst.greedy_host(3)
        np.testing.assert_array_equal(np.concatenate([a, b, c]), r1[0])
        np.testing.assert_array_equal(np.concatenate([fa, fb, fc]), r1[1])
        inst.set_lazy(True)
        inst.reset()
        d, fd = inst.greedy_host(12)
        np.testing.assert_array_equal(d, r1[0])
        np.testing.assert_array_equal(fd, r1[1])
        inst.reload(V2)
        e, fe = inst.greedy_host(12)
        np.testing.assert_array_equal(e, r2[0])
        np.testing.assert_array_equal(fe, r2[1])


def test_lazy_fp32_precision_runs_full_rounds(torch):
    V = gmm(3000, 16, 3)
    with ebc.Instance(V, precision="fp32") as a, ebc.Instance(V, precision="fp32", lazy=True) as b:
        ia, fa = a.greedy_host(6)
        ib, fb = b.greedy_host(6)
        assert b.stats()["bulk_candidates"] == 0
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(fa, fb)


def test_lazy_regime_workload_sampled(torch):
    """Drifting-regime features (the headline generator) at n=60,000, d=128,
    k=40: lazy equals full bitwise and evaluates a fraction of the candidates."""
    V = synth.regime_greedy(seed=1, n=60_000, d=128, k=40)["V"]
    (ia, fa), (ib, fb), st = full_and_lazy(V, 40, "bf16")
    np.testing.assert_array_equal(ib, ia)
    np.testing.assert_array_equal(fb, fa)
    full = sum(60_000 - t for t in range(40))
    print("regime n=60k: bulk candidates", st["bulk_candidates"], "of", full, f"({st['bulk_candidates'] / full:.3%})")
    assert st["bulk_candidates"] < 0.5 * full


def test_batch_lazy_equals_alone(torch):
    rng = np.random.default_rng(8)
    specs = []
    for n, d in [(3000, 33), (12000, 64), (800, 128), (7000, 16)]:
        specs.append((gmm(n, d, int(rng.integers(1 << 30))), int(rng.integers(3, 13))))
    with ebc.Batch(max_slots=3, budget_bytes=8 << 30) as b:
        b.set_lazy(True)
        tickets = [b.submit(V, k, "bf16") for V, k in specs]
        b.run()
        got = [b.poll(t) for t in tickets]
    for (V, k), (idx, f) in zip(specs, got):
        with ebc.Instance(V, precision="bf16") as inst:
            ridx, rf = inst.greedy_host(k)
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)
