"""Pins of the oracle's threshold sieve (the streaming optimisers the paper
names beside Greedy: Sec. 2, Sec. 4.1; Three Sieves in the case study of
Sec. 6, Fig. 4) against values fixed without it: hand-worked decisions
(tests/golden/sieve_examples.json), closed forms, the definitional discrete
derivative (Sec. 3, Def. 1) computed from scratch with Algorithm 1, and the
approximation guarantees that follow from submodularity, checked against
the brute-force optimum."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sieve_examples.json")


def _gold():
    with open(GOLD) as fh:
        return json.load(fh)


def _start(V, S):
    m = oracle.norms(V)
    sel = np.zeros(V.shape[0], dtype=np.uint8)
    for c in S:
        oracle.update_m(V, m, c)
        sel[c] = 1
    return m, sel


@pytest.mark.parametrize("ex", _gold()["examples"], ids=lambda e: e["name"])
def test_hand_worked_sieve(ex):
    V = np.array(_gold()["V"], dtype=np.float32)
    m, sel = _start(V, ex["start_S"])
    r = oracle.sieve(V, ex["stream"], ex["K"], ex["thr"], ex["patience"], m=m, selected=sel,
                     f_start=ex["f_start"])
    assert r["idx"].tolist() == ex["idx"]
    assert r["f"].tolist() == ex["f"]            # dyadic values: exact
    assert r["level"] == ex["level"] and r["rejections"] == ex["rejections"]
    dec = ex["decided"]
    np.testing.assert_allclose(r["margin"][:dec], ex["margin"], rtol=0, atol=1e-15)
    assert np.all(np.isnan(r["margin"][dec:]))


def _rand(n, d, seed):
    return synth.zscore_to_f32(np.random.default_rng(seed).standard_normal((n, d)))


def test_zero_threshold_takes_the_first_K_unselected():
    """v = 0 gives tau = -f(S)/(K - |S|) <= 0: every item not in S is taken
    until |S| = K, and f is f of those items (form A and form B)."""
    V = _rand(30, 3, 1)
    m, sel = _start(V, [4, 7])
    stream = [7, 3, 3, 4, 11, 0, 5, 9]
    f0 = oracle.f(V, [4, 7])
    r = oracle.sieve(V, stream, 6, [0.0], 0, m=m, selected=sel, f_start=f0)
    assert r["idx"].tolist() == [3, 11, 0, 5]
    S = [4, 7, 3, 11, 0, 5]
    assert r["f_end"] == pytest.approx(oracle.f_alg1(V, S), rel=1e-12)
    assert r["f_end"] == pytest.approx(oracle.f(V, S), rel=1e-12)
    assert np.isnan(r["margin"][7])              # |S| = K after position 6


def test_unreachable_threshold_rejects_and_walks_the_levels():
    """tau = v / (2K) above the largest singleton gain (<= L0): nothing is
    taken, the level moves every `patience` rejections and stops at the last."""
    V = _rand(40, 4, 2)
    L0 = float(np.mean(oracle.norms(V)))
    thr = [1e3 * L0 * (5 - j) for j in range(5)]
    for T, length in [(3, 10), (4, 40), (1, 3), (7, 6)]:
        r = oracle.sieve(V, np.arange(length) % 40, 3, thr, T)
        assert r["idx"].size == 0
        assert r["level"] == min(length // T, len(thr) - 1)
        reached_last = length // T >= len(thr) - 1
        if not reached_last:
            assert r["rejections"] == length % T
    r = oracle.sieve(V, np.arange(40), 3, thr, 0)
    assert r["level"] == 0 and r["rejections"] == 40


@pytest.mark.parametrize("seed", range(6))
def test_decisions_follow_the_definitional_derivative(seed):
    """Every decision agrees with Delta_f(e|S) = f(S u {e}) - f(S) recomputed
    from scratch by Algorithm 1 (no per-point minimum carried over)."""
    rng = np.random.default_rng(seed)
    n, K = 24, 5
    V = _rand(n, 3, 100 + seed)
    stream = rng.permutation(n)
    m1 = float(oracle.greedy(V, 1)[1][0])
    thr = oracle.threshold_ladder(m1, K, 0.3, 1.0)
    T = 3
    r = oracle.sieve(V, stream, K, thr, T)
    S, lev, rej = [], 0, 0
    fS = 0.0
    for p, e in enumerate(stream):
        if len(S) == K:
            assert np.isnan(r["margin"][p])
            continue
        if e in S:
            take = False
        else:
            tau = (thr[lev] / 2.0 - fS) / (K - len(S))
            delta = oracle.f_alg1(V, S + [int(e)]) - oracle.f_alg1(V, S)
            if r["margin"][p] > 1e-9:
                take = delta >= tau
            else:
                take = int(e) in r["idx"].tolist()
        if take:
            S.append(int(e))
            fS = oracle.f_alg1(V, S)
            rej = 0
        else:
            rej += 1
            if rej >= T:
                lev = min(lev + 1, len(thr) - 1)
                rej = 0
    assert r["idx"].tolist() == S
    assert r["f_end"] == pytest.approx(oracle.f_alg1(V, S), rel=1e-12)
    np.testing.assert_allclose(r["f"], [oracle.f_alg1(V, S[:j + 1]) for j in range(len(S))], rtol=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_single_threshold_guarantees_against_brute_force(seed):
    """For one fixed threshold v over a stream holding all of V:
    f(S_j) >= (v/2) j / K after every acceptance; a full summary has
    f >= v/2; otherwise f > OPT_K - v/2 (each rejected optimum element adds
    less than v/(2K) by submodularity).  Sieve Streaming's best sieve reaches
    (1 - eps) OPT_K / 2."""
    rng = np.random.default_rng(seed)
    n, K, eps = 11, 2 + seed % 3, 0.25
    V = _rand(n, 2 + seed % 4, 200 + seed)
    opt, _ = oracle.exhaustive_opt(V, K)
    m1 = float(oracle.greedy(V, 1)[1][0])
    stream = rng.permutation(n)
    best, allr, thr = oracle.sieve_streaming(V, stream, K, eps, m1)
    assert np.all(np.diff(thr) < 0) and thr[-1] >= m1 and thr[0] <= 2 * K * m1
    assert thr[-1] / (1 + eps) < m1 and thr[0] * (1 + eps) > 2 * K * m1
    tol = 1e-12 * max(opt, 1.0)
    for v, r in zip(thr, allr):
        for j, fj in enumerate(r["f"]):
            assert fj >= v / 2 * (j + 1) / K - tol
        if r["idx"].size == K:
            assert r["f_end"] >= v / 2 - tol
        else:
            assert r["f_end"] > opt - v / 2 - tol
    assert best["f_end"] >= (1 - eps) * opt / 2 - tol
    assert best["f_end"] == max(r["f_end"] for r in allr)


@pytest.mark.parametrize("seed", range(4))
def test_three_sieves_full_summary_reaches_half_the_final_threshold(seed):
    """Thresholds only decrease, so every acceptance met the rule for the
    final threshold too: a full summary has f >= v_final / 2."""
    rng = np.random.default_rng(seed)
    n, K = 60, 6
    V = _rand(n, 3, 300 + seed)
    m1 = float(oracle.greedy(V, 1)[1][0])
    for T in (1, 4, 20):
        r = oracle.three_sieves(V, rng.permutation(n), K, 0.2, T, m1)
        thr = oracle.threshold_ladder(m1, K, 0.2, 1.0)
        if r["idx"].size == K:
            assert r["f_end"] >= thr[r["level"]] / 2 * (1 - 1e-12)
        assert len(set(r["idx"].tolist())) == r["idx"].size


def test_stream_in_pieces_equals_one_pass():
    V = _rand(80, 3, 9)
    m1 = float(oracle.greedy(V, 1)[1][0])
    thr = oracle.threshold_ladder(m1, 8, 0.1, 1.0)
    stream = np.random.default_rng(3).permutation(80)
    one = oracle.sieve(V, stream, 8, thr, 5)
    m, sel = _start(V, [])
    f, lev, rej, idx = 0.0, 0, 0, []
    for a, b in [(0, 7), (7, 8), (8, 40), (40, 80)]:
        r = oracle.sieve(V, stream[a:b], 8, thr, 5, m=m, selected=sel, f_start=f, level=lev, rejections=rej)
        f, lev, rej = r["f_end"], r["level"], r["rejections"]
        idx += r["idx"].tolist()
    assert idx == one["idx"].tolist()
    assert f == one["f_end"] and lev == one["level"] and rej == one["rejections"]


def test_ladder_closed_form():
    # (1+eps)^i for eps = 1: powers of two in [m, upper K m]
    np.testing.assert_array_equal(oracle.threshold_ladder(3.0, 4, 1.0, 2.0), [16.0, 8.0, 4.0])
    np.testing.assert_array_equal(oracle.threshold_ladder(1.0, 1, 1.0, 1.0), [1.0])
    t = oracle.threshold_ladder(0.37, 50, 0.05, 1.0)
    i = np.round(np.log(t) / math.log(1.05))
    assert np.all(np.diff(i) == -1) and t[-1] >= 0.37 and t[0] <= 50 * 0.37


def test_sieve_errors():
    V = _rand(5, 2, 0)
    with pytest.raises(oracle.OracleError):
        oracle.sieve(V, [0, 5], 2, [1.0], 0)      # index outside [0, n)
    with pytest.raises(oracle.OracleError):
        oracle.sieve(V, [0], 6, [1.0], 0)         # K > n
    with pytest.raises(oracle.OracleError):
        oracle.sieve(V, [0], 2, [1.0], 0, level=1)
