"""Seeded input generators: reproducible, right shapes, z-scored."""
import numpy as np

from paper_2105_12026_gb300 import synth


def test_reproducible_and_seed_sensitive():
    a = synth.plain_greedy_small(seed=0)["V"]
    b = synth.plain_greedy_small(seed=0)["V"]
    c = synth.plain_greedy_small(seed=1)["V"]
    assert a.dtype == np.float32 and a.shape == (1000, 16)
    assert synth.digest(a) == synth.digest(b)
    assert synth.digest(a) != synth.digest(c)


def test_zscore_population_moments():
    V = synth.plain_greedy_small(seed=2)["V"].astype(np.float64)
    np.testing.assert_allclose(V.mean(0), 0.0, atol=1e-6)
    np.testing.assert_allclose(V.std(0), 1.0, rtol=1e-6)


def test_zscore_constant_dimension_stays_zero():
    x = np.ones((10, 3))
    x[:, 1] = np.arange(10)
    z = synth.zscore_to_f32(x)
    assert (z[:, 0] == 0).all() and (z[:, 2] == 0).all()


def test_multiset_sets_are_valid():
    w = synth.multiset_eval(seed=0, n=2000, d=8, l=50)
    idx, off = w["idx"], w["off"]
    assert off[0] == 0 and off.size == 51 and (np.diff(off) >= 1).all() and (np.diff(off) <= 64).all()
    assert idx.min() >= 0 and idx.max() < 2000
    for j in range(50):
        s = idx[off[j]:off[j + 1]]
        assert len(set(s.tolist())) == s.size  # without replacement


def test_drift_regimes_outliers():
    rng = np.random.default_rng(0)
    x = synth.drift_regimes(rng, 6000, 16)
    assert x.shape == (6000, 16)


def test_instance_mix_ranges():
    mix = synth.instance_mix(seed=0)
    assert len(mix) == 256
    assert all(2000 <= s.n <= 100_000 for s in mix)
    assert all(s.d in (16, 32, 64, 128) for s in mix)
    assert all(5 <= s.k <= 50 for s in mix)
    assert all(4 <= s.clusters <= 64 for s in mix)


def test_request_trace_rate():
    tr = synth.request_trace(seed=0, rate=50.0, horizon_s=20.0)
    assert 800 < len(tr) < 1200
    assert all(a.t_arrive <= b.t_arrive for a, b in zip(tr, tr[1:]))
    assert any(r.large for r in tr)


def test_case_study_series_shape_and_regimes():
    a = synth.case_study_series(seed=3, n=300, d=500)
    b = synth.case_study_series(seed=3, n=300, d=500)
    assert a.shape == (300, 500) and a.dtype == np.float32
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(a.mean(0), 0.0, atol=1e-4)
    np.testing.assert_allclose(a.std(0), 1.0, atol=1e-3)
    # contiguous runs of a regime: neighbouring cycles are far more alike than random pairs
    near = np.mean(np.sum((a[1:] - a[:-1]) ** 2, 1))
    far = np.mean(np.sum((a[np.random.default_rng(0).permutation(300)] - a) ** 2, 1))
    assert near < 0.5 * far
