"""Autotuner of the bulk kernel (ebc_autotune): it stores one entry per
(precision, padded d, n bucket), later launches use it, and neither the
search nor the tuned configuration changes picks or f (bitwise)."""
import numpy as np
import pytest

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


def gmm(n, d, seed):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, 8, sigma=None))


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp8"])
def test_autotune_keeps_results(torch, prec, tmp_path):
    ebc.ebc_tune_clear()
    V = gmm(9000, 64, 3)
    with ebc.Instance(V, precision=prec) as a:
        ia, fa = a.greedy_host(6)
    with ebc.Instance(V, precision=prec) as b:
        b.greedy_host(2)  # state mid-run: the search must leave it alone
        b.autotune(2)
        assert ebc.ebc_tune_count() == 1
        ib, fb = b.greedy_host(4)
    np.testing.assert_array_equal(np.concatenate([ia[:2], ib]), ia)
    np.testing.assert_array_equal(fb, fa[2:])
    with ebc.Instance(V, precision=prec) as c:  # a new handle in the bucket uses the entry
        ic, fc = c.greedy_host(6)
    np.testing.assert_array_equal(ic, ia)
    np.testing.assert_array_equal(fc, fa)
    path = tmp_path / "tune.json"
    ebc.ebc_tune_save(str(path))
    ebc.ebc_tune_clear()
    ebc.ebc_tune_load(str(path))
    assert ebc.ebc_tune_count() == 1
    ebc.ebc_tune_clear()


def test_autotune_rejects_fp32_and_bad_reps(torch):
    V = gmm(500, 16, 1)
    with ebc.Instance(V) as inst:
        with pytest.raises(ebc.EbcError) as ei:
            inst.autotune(2)
        assert ei.value.status == ebc.EBC_EINVAL
        inst.set_precision("bf16")
        with pytest.raises(ebc.EbcError):
            inst.autotune(0)


def test_batch_autotune_equals_alone(torch):
    ebc.ebc_tune_clear()
    specs = [(gmm(3000, 32, 11), 5), (gmm(3500, 32, 12), 4), (gmm(12000, 128, 13), 3)]
    with ebc.Batch(max_slots=2) as b:
        b.set_autotune(1)
        tickets = [b.submit(V, k, "bf16") for V, k in specs]
        b.run()
        got = [b.poll(t) for t in tickets]
    assert ebc.ebc_tune_count() == 2  # buckets (bf16, 64, 11) and (bf16, 128, 13)
    for (V, k), (idx, f) in zip(specs, got):
        with ebc.Instance(V, precision="bf16") as inst:
            ridx, rf = inst.greedy_host(k)
        np.testing.assert_array_equal(idx, ridx)
        np.testing.assert_array_equal(f, rf)
    ebc.ebc_tune_clear()
