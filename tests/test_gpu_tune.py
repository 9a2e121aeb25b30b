"""Autotuner of the bulk kernel (ebc_autotune): it stores one entry per
(precision, padded d, n bucket), later launches use it, and neither the
search nor the tuned configuration changes picks or f (bitwise).  Tile
shapes forced through a table entry (128-point tiles, MMA issuer turns)
give the default's raw gains (up to FP32 summation order at 128 points) and
the same picks and f."""
import json
import math

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
        ent = b.tune_entry()
        assert ent is not None and ent["bn"] in (128, 256) and ent["ms"] > 0
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


def _row_bytes(prec, d):
    if prec == "fp8":
        return (d + 127) // 128 * 128
    return 2 * ((d + 63) // 64 * 64)


def _force_entry(tmp_path, prec, d, n, **cfg):
    """Load a tuning-table entry for (prec, d, n)'s bucket with the given shape."""
    ent = {"prec": ebc.PRECISIONS[prec], "rb": _row_bytes(prec, d), "nbucket": int(math.floor(math.log2(n)))}
    ent.update(cfg)
    path = tmp_path / "forced.json"
    path.write_text(json.dumps({"version": 1, "entries": [ent]}))
    ebc.ebc_tune_load(str(path))


@pytest.mark.parametrize("prec,d,na,ns,chunk,bn,turns,es", [
    ("bf16", 128, 1, 4, 0, 128, -1, 0), ("bf16", 128, 2, 2, 1, 128, -1, 0), ("fp16", 40, 2, 6, 0, 128, -1, 0),
    ("fp8", 128, 2, 6, 2, 128, -1, 0), ("bf16", 64, 1, 3, 0, 128, -1, 0),
    ("bf16", 128, 1, 2, 0, 256, 0, 0), ("bf16", 64, 2, 3, 0, 256, 1, 0), ("fp8", 128, 2, 2, 1, 256, 1, 0),
    ("bf16", 128, 1, 2, 0, 256, 1, 1), ("bf16", 64, 2, 3, 0, 256, 0, 1), ("fp8", 128, 2, 3, 0, 256, -1, 1),
    ("fp16", 40, 1, 4, 2, 256, 0, 1)])
def test_tile_shapes_match_default(torch, prec, d, na, ns, chunk, bn, turns, es, tmp_path):
    """A forced table entry: 128-point tiles and the other drain split give
    the default's raw gains up to FP32 summation order; issuer turns on or
    off give them bitwise (each region's MMA sequence is the same); picks
    and f are always bitwise."""
    n = 5037  # 20 tiles of 256 / 40 of 128 after padding, ragged tail
    V = gmm(n, d, 21)
    cand = np.random.default_rng(5).choice(n, 700, replace=False).astype(np.int32)
    ebc.ebc_tune_clear()
    try:
        with ebc.Instance(V, precision=prec) as a:
            assert a.tune_entry() is None
            g0 = a.gains_host()
            l0 = a.gains_host(cand)
            i0, f0 = a.greedy_host(8)
        _force_entry(tmp_path, prec, d, n, bn=bn, na=na, ns=ns, chunk=chunk, turns=turns, es=es)
        with ebc.Instance(V, precision=prec) as b:
            assert b.tune_entry() == {"bn": bn, "na": na, "ns": ns, "chunk": chunk, "turns": turns, "es": es,
                                      "ms": 0.0}
            g1 = b.gains_host()
            l1 = b.gains_host(cand)
            i1, f1 = b.greedy_host(8)
            st = b.stats()
    finally:
        ebc.ebc_tune_clear()
    default_es = 1 if _row_bytes(prec, d) <= 128 else 0  # the library's default drain split
    if bn == 256 and chunk == 0 and es == default_es:
        np.testing.assert_array_equal(g1, g0)
        np.testing.assert_array_equal(l1, l0)
    else:
        # the same FP32 terms summed in another grouping (64 instead of 128
        # per thread and tile, or other V chunks, in FP64)
        scale = float(np.max(np.abs(g0)))
        np.testing.assert_allclose(g1, g0, rtol=2e-6, atol=1e-9 * scale)
        np.testing.assert_allclose(l1, l0, rtol=2e-6, atol=1e-9 * scale)
    np.testing.assert_allclose(l1, g1[cand], rtol=2e-6, atol=1e-9 * float(np.max(np.abs(g1))))
    np.testing.assert_array_equal(i1, i0)
    np.testing.assert_array_equal(f1, f0)
    assert st["rounds"] == 8


def test_autotune_128_point_entry_roundtrip(torch, tmp_path):
    """An entry with 128-point tiles survives save / load with its width."""
    ebc.ebc_tune_clear()
    _force_entry(tmp_path, "bf16", 128, 30000, bn=128, na=1, ns=4, chunk=0)
    out = tmp_path / "out.json"
    ebc.ebc_tune_save(str(out))
    ebc.ebc_tune_clear()
    ebc.ebc_tune_load(str(out))
    V = gmm(30000, 128, 2)
    with ebc.Instance(V, precision="bf16") as inst:
        assert inst.tune_entry()["bn"] == 128
    ebc.ebc_tune_clear()
