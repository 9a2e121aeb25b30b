"""Threshold sieve over a stream (ebc_sieve_host; the streaming optimisers of
Sec. 2 / Sec. 4.1, Three Sieves in the case study of Sec. 6) against the
FP64 oracle.

Decisions compare exact gains with tau = (v/2 - f(S)) / (K - |S|); the GPU
takes them on certified gains (bulk upper bounds reject, the exact gain
decides), so the accepted items must be the oracle's up to the first stream
position whose decision the oracle itself sees within 1e-6 relative of a
tie; f values match at F_RTOL.  At the full headline size (n = 200,000,
d = 128) the accepted items and a sample of rejected ones are re-decided by
the oracle under the GPU's own summary prefix.
"""
import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import ebc, synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-7
TIE = 1e-6


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


def compare(stream, ref, idx, f):
    """Accepted items equal up to the oracle's first near-tie decision; f of
    the common prefix within F_RTOL; returns the compared prefix length."""
    pos = {int(e): p for p, e in enumerate(stream)}
    ties = np.nonzero(ref["margin"] <= TIE)[0]
    cut = int(ties[0]) if ties.size else len(stream)
    ra = [e for e in ref["idx"].tolist() if pos[e] < cut]
    ga = [e for e in idx.tolist() if pos[e] < cut]
    assert ga == ra, (ga[:20], ra[:20], cut)
    j = len(ra)
    np.testing.assert_allclose(f[:j], ref["f"][:j], rtol=F_RTOL)
    if cut == len(stream):
        assert idx.tolist() == ref["idx"].tolist()
    return j, cut


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32", "fp8"])
@pytest.mark.parametrize("n,d,K,T", [(2000, 16, 12, 40), (1500, 64, 20, 25), (777, 100, 9, 10),
                                     (2500, 128, 15, 100), (300, 5, 40, 3), (900, 300, 10, 15)])
def test_three_sieves_matches_oracle(torch, prec, n, d, K, T):
    if prec == "fp8" and d > 128:
        pytest.skip("the FP8 path holds d <= 128")
    V = gmm(n, d, 7 * n + d)
    stream = np.random.default_rng(n + d).permutation(n).astype(np.int32)
    m1 = float(oracle.greedy(V, 1)[1][0])
    ref = oracle.three_sieves(V, stream, K, 0.1, T, m1)
    with ebc.Instance(V, precision=prec) as inst:
        idx, f, sv = ebc.three_sieves(inst, stream, K, 0.1, T, m1)
        assert inst.current_f() == pytest.approx(f[-1] if f.size else 0.0, rel=1e-9, abs=1e-12)
    j, cut = compare(stream, ref, idx, f)
    if cut == n:
        assert sv.level == ref["level"] and sv.rejections == ref["rejections"]
    c = sv.counters()
    assert c["bounded"] >= 1 and c["exact"] >= idx.size
    print(prec, n, d, K, T, "accepted", idx.size, "compared", j, "bounded", c["bounded"], "exact", c["exact"])


def test_sieve_streaming_matches_oracle(torch):
    n, d, K, eps = 1200, 32, 8, 0.2
    V = gmm(n, d, 5)
    stream = np.random.default_rng(1).permutation(n).astype(np.int32)
    m1 = float(oracle.greedy(V, 1)[1][0])
    rbest, rall, rthr = oracle.sieve_streaming(V, stream, K, eps, m1)
    with ebc.Instance(V, precision="bf16") as inst:
        idx, f, ends, thr = ebc.sieve_streaming(inst, stream, K, eps, m1)
        np.testing.assert_array_equal(thr, rthr)
        for v, e, r in zip(thr, ends, rall):
            if np.all(r["margin"][~np.isnan(r["margin"])] > TIE):
                assert e == pytest.approx(r["f_end"], rel=F_RTOL), v
        assert inst.current_f() == pytest.approx(max(ends), rel=1e-9)
    assert max(ends) == pytest.approx(rbest["f_end"], rel=F_RTOL)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32", "fp8"])
def test_gain_bounds_are_upper_bounds(torch, prec):
    """ebc_gain_bounds against the oracle's exact gains, at S = {} and after
    a few Greedy picks: every bound >= the exact gain, and close to it."""
    n, d = 1500, 40
    V = gmm(n, d, 14)
    cand = np.arange(0, n, 3, dtype=np.int32)
    m = oracle.norms(V)
    with ebc.Instance(V, precision=prec) as inst:
        for step in range(2):
            ub = inst.gain_bounds_host(cand)
            ex = oracle.gains(V, m, cand)
            assert np.all(ub >= ex * (1 - 1e-12)), np.min(ub - ex)
            assert np.all(ub <= ex + 0.05 * max(ex.max(), 1e-9))
            picks, _ = inst.greedy_host(4)
            for c in picks:
                oracle.update_m(V, m, c)
                ex_sel = oracle.gains(V, m, [c])
                assert ex_sel[0] == 0.0
        assert np.all(inst.gain_bounds_host(picks) == 0.0)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_primed_bounds_and_cache_keep_decisions(torch, prec):
    """Singleton bounds as the sieve's starting bounds, and the bounds the
    handle keeps across calls, change the work but not one decision."""
    n, d, K = 2500, 32, 15
    V = gmm(n, d, 19)
    stream = np.random.default_rng(9).permutation(n).astype(np.int32)
    with ebc.Instance(V, precision=prec) as a:
        m1 = a.max_singleton()
        thr = ebc.ebc_threshold_ladder(m1, K, 0.05, 1.0)
        plain = a.sieve(K, thr, 40)
        i1, f1 = plain.feed(stream)
        a.reset()
        primed = a.sieve(K, thr, 40, bounds=a.singleton_bounds())
        i2, f2 = primed.feed(stream)
        a.reset()                                   # the kept bounds are dropped
        again = a.sieve(K, thr, 40)
        i3, f3 = again.feed(stream)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(i1, i3)
    np.testing.assert_array_equal(f1, f3)
    assert primed.counters()["bounded"] <= plain.counters()["bounded"]
    assert again.counters()["bounded"] == plain.counters()["bounded"]


def test_sieve_streaming_workers_equal_sequential(torch):
    n, d, K, eps = 3000, 48, 10, 0.15
    V = gmm(n, d, 8)
    stream = np.random.default_rng(6).permutation(n).astype(np.int32)
    with ebc.Instance(V, precision="bf16") as a:
        m1 = a.max_singleton()
        i1, f1, e1, t1 = ebc.sieve_streaming(a, stream, K, eps, m1)
        fa = a.current_f()
    with ebc.Instance(V, precision="bf16") as b:
        i4, f4, e4, t4 = ebc.sieve_streaming(b, stream, K, eps, m1, workers=4, V=V)
        fb = b.current_f()
    np.testing.assert_array_equal(t1, t4)
    assert e1 == e4
    np.testing.assert_array_equal(i1, i4)
    np.testing.assert_array_equal(f1, f4)
    assert fa == fb


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_stream_in_pieces_equals_one_pass(torch, prec):
    V = gmm(3000, 48, 21)
    stream = np.random.default_rng(2).permutation(3000).astype(np.int32)
    m1 = float(oracle.greedy(V, 1)[1][0])
    thr = ebc.ebc_threshold_ladder(m1, 25, 0.05, 1.0)
    with ebc.Instance(V, precision=prec) as a:
        one = a.sieve(25, thr, 30)
        i1, f1 = one.feed(stream)
    with ebc.Instance(V, precision=prec) as b:
        sv = b.sieve(25, thr, 30)
        for lo, hi in [(0, 1), (1, 2), (2, 100), (100, 101), (101, 2000), (2000, 3000)]:
            sv.feed(stream[lo:hi])
    assert sv.idx == i1.tolist()
    np.testing.assert_array_equal(np.array(sv.f), f1)
    assert (sv.level, sv.rejections) == (one.level, one.rejections)


def test_continues_from_greedy_state_with_selected_and_duplicate_items(torch):
    """Sieve after 3 Greedy picks: items already in S (and repeats in the
    stream) are rejections; the oracle runs from the same state."""
    n, d = 900, 24
    V = gmm(n, d, 33)
    rng = np.random.default_rng(4)
    ridx, rf, _ = oracle.greedy(V, 3)
    m = oracle.norms(V)
    sel = np.zeros(n, dtype=np.uint8)
    for c in ridx:
        oracle.update_m(V, m, c)
        sel[c] = 1
    stream = np.concatenate([ridx[:2], rng.integers(0, n, 600), ridx[2:], rng.integers(0, n, 300)]).astype(np.int32)
    m1 = float(oracle.greedy(V, 1)[1][0])
    thr = oracle.threshold_ladder(m1, 14, 0.1, 1.0)
    ref = oracle.sieve(V, stream, 14, thr, 20, m=m, selected=sel, f_start=float(rf[-1]))
    with ebc.Instance(V, precision="bf16") as inst:
        gi, gf = inst.greedy_host(3)
        np.testing.assert_array_equal(gi, ridx)
        sv = inst.sieve(14, thr, 20)
        idx, f = sv.feed(stream)
    ties = np.nonzero(ref["margin"] <= TIE)[0]
    if ties.size == 0:
        assert idx.tolist() == ref["idx"].tolist()
        assert (sv.level, sv.rejections) == (ref["level"], ref["rejections"])
    np.testing.assert_allclose(f[:2], ref["f"][:2], rtol=F_RTOL)
    assert not set(idx.tolist()) & set(ridx.tolist())


def test_edge_cases(torch):
    V = gmm(400, 8, 2)
    with ebc.Instance(V, precision="bf16") as inst:
        # empty stream and a summary already full: nothing decided
        sv = inst.sieve(3, [1.0], 0)
        assert sv.feed(np.zeros(0, dtype=np.int32))[0].size == 0
        inst.greedy_host(3)
        full = inst.sieve(3, [0.0], 0)
        assert full.feed(np.arange(10))[0].size == 0 and full.state.consumed == 0
        inst.reset()
        # v = 0: tau <= 0 takes the first K items not in S
        z = inst.sieve(4, [0.0], 0)
        idx, f = z.feed(np.array([5, 5, 9, 1, 7, 3], dtype=np.int32))
        assert idx.tolist() == [5, 9, 1, 7] and z.state.consumed == 5
        assert f[-1] == pytest.approx(oracle.f(V, [5, 9, 1, 7]), rel=1e-9)
        # argument errors leave the state alone
        before = (z.level, z.rejections, inst.current_f())
        with pytest.raises(ebc.EbcError):
            z.feed(np.array([1, 400], dtype=np.int32))
        bad = inst.sieve(5, [np.inf], 0)
        with pytest.raises(ebc.EbcError):
            bad.feed(np.array([1], dtype=np.int32))
        over = inst.sieve(401, [1.0], 0)
        with pytest.raises(ebc.EbcError):
            over.feed(np.array([1], dtype=np.int32))
        assert (z.level, z.rejections, inst.current_f()) == before


def test_headline_size_sampled(torch):
    """Three Sieves over the drifting-regime features (n = 200,000, d = 128,
    K = 100, stream in time order) at BF16: every accepted item and a sample
    of rejected ones re-decided by the oracle under the GPU's summary prefix
    and threshold schedule."""
    n, d, K, eps, T = 200_000, 128, 100, 0.01, 2000
    V = synth.regime_greedy(seed=0, n=n, d=d, k=K)["V"]
    stream = np.arange(n, dtype=np.int32)
    with ebc.Instance(V, precision="bf16") as inst:
        m1 = inst.max_singleton()
        thr = ebc.ebc_threshold_ladder(m1, K, eps, 1.0)
        sv = inst.sieve(K, thr, T)
        idx, f = sv.feed(stream)
        c = sv.counters()
    assert 0 < idx.size <= K and len(set(idx.tolist())) == idx.size
    assert np.all(np.diff(idx) > 0)                   # accepted in stream order
    # replay the schedule from the accept positions (stream position = item)
    acc = set(idx.tolist())
    end = c["consumed"]
    level_at = np.zeros(end, dtype=np.int64)
    lev = rej = 0
    for p in range(end):
        level_at[p] = lev
        if p in acc:
            rej = 0
        else:
            rej += 1
            if rej >= T:
                lev = min(lev + 1, thr.size - 1)
                rej = 0
    assert (lev, rej) == (sv.level, sv.rejections)
    rng = np.random.default_rng(0)
    rejected = np.setdiff1d(np.arange(end), idx)
    probe = np.sort(rng.choice(rejected, size=min(40, rejected.size), replace=False))
    m = oracle.norms(V)
    fS, s, a = 0.0, 0, 0
    checked = 0
    for p in sorted(set(probe.tolist()) | acc):
        while a < idx.size and idx[a] < p:           # summary prefix before p
            fS = float(f[a])
            oracle.update_m(V, m, int(idx[a]))
            a += 1
            s += 1
        tau = (thr[level_at[p]] / 2.0 - fS) / (K - s)
        g = float(oracle.gains(V, m, [p])[0])
        if p in acc:                                 # f after accepting p: prefix f + exact gain
            assert f[a] == pytest.approx(fS + g, rel=F_RTOL)
        if abs(g - tau) > TIE * max(abs(g), abs(tau)):
            assert (g >= tau) == (p in acc), (p, g, tau)
            checked += 1
    assert np.all(np.diff(f) >= 0)
    assert checked >= idx.size // 2
    print("accepted", idx.size, "consumed", end, "bounded", c["bounded"], "exact", c["exact"], "f", f[-1])
