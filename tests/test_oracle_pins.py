"""Pins for the CPU oracle, independent of the oracle itself.

Each check compares the oracle with something the paper or mathematics fixes:
hand-worked fixtures (tests/golden/hand_examples.json), closed forms,
invariants of monotone submodular functions (Sec. 3, Def. 2 and 3), the
(1 - 1/e) Greedy guarantee against exhaustive search (Sec. 3), an
independent library route (torch.cdist in FP64), and agreement between the
oracle's two independently written forms of f (Algorithm 1 vs the relu form).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _examples():
    with open(GOLDEN) as fh:
        return json.load(fh)["examples"]


@pytest.mark.parametrize("ex", _examples(), ids=lambda e: e["name"])
def test_hand_examples_f(ex):
    V = np.asarray(ex["V"], dtype=np.float32)
    np.testing.assert_array_equal(oracle.norms(V), np.asarray(ex["norms"], dtype=np.float64))
    assert oracle.loss(V, [], with_e0=True) == pytest.approx(ex["L0"], rel=1e-15)
    for S, fv in zip(ex["sets"], ex["f"]):
        assert oracle.f(V, S) == pytest.approx(fv, rel=1e-14, abs=1e-15), S
        assert oracle.f_alg1(V, S) == pytest.approx(fv, rel=1e-14, abs=1e-14), S
    idx = np.asarray([0] * 0, dtype=np.int32)
    off = np.zeros(len(ex["sets"]) + 1, dtype=np.int64)
    members = []
    for j, S in enumerate(ex["sets"]):
        members.extend(S)
        off[j + 1] = len(members)
    idx = np.asarray(members, dtype=np.int32)
    np.testing.assert_allclose(oracle.eval_sets(V, idx, off), ex["f"], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("ex", _examples(), ids=lambda e: e["name"])
def test_hand_examples_greedy(ex):
    V = np.asarray(ex["V"], dtype=np.float32)
    idx, fv, gap = oracle.greedy(V, ex["greedy_k"])
    assert idx.tolist() == ex["greedy_idx"]
    np.testing.assert_allclose(fv, ex["greedy_f"], rtol=1e-14)
    np.testing.assert_allclose(gap, ex["greedy_gap"], rtol=1e-12, atol=1e-15)


def test_loss_without_e0_empty_is_float_max():
    # Algorithm 1 starts the running minimum at the largest float value.
    V = np.ones((3, 2), np.float32)
    assert oracle.loss(V, [], with_e0=False) == np.finfo(np.float64).max


def _rand(n, d, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d)).astype(np.float32)


def test_closed_forms():
    V = _rand(37, 5, 1)
    nv = (V.astype(np.float64) ** 2).sum(1)
    # f(empty) = 0
    assert oracle.f(V, []) == 0.0
    assert oracle.f_alg1(V, []) == 0.0
    # f(V) = L({e0}) = mean |v|^2: every v covers itself at distance 0
    assert oracle.f(V, np.arange(37)) == pytest.approx(nv.mean(), rel=1e-14)
    # n = 1: f({v}) = |v|^2
    assert oracle.f(V[:1], [0]) == pytest.approx(nv[0], rel=1e-15)
    # distance to self is zero, symmetric, matches a hand sum
    assert oracle.sqdist(V[3], V[3]) == 0.0
    assert oracle.sqdist(V[3], V[4]) == oracle.sqdist(V[4], V[3])
    x = np.array([1.5, -2.0, 0.25], np.float32)
    y = np.array([0.5, 1.0, 0.25], np.float32)
    assert oracle.sqdist(x, y) == 1.0 + 9.0 + 0.0


def test_zscore_gives_L0_equal_d():
    # after a population z-score every dimension has mean 0 and variance 1,
    # so L({e0}) = mean_v |v|^2 = sum_i var_i = d (up to the FP32 cast)
    V = synth.plain_greedy_small(seed=3)["V"]
    L0 = oracle.loss(V, [], with_e0=True)
    assert L0 == pytest.approx(V.shape[1], rel=1e-6)
    assert oracle.f(V, np.arange(V.shape[0])) == pytest.approx(V.shape[1], rel=1e-6)


def test_two_forms_agree():
    V = _rand(300, 7, 2)
    rng = np.random.default_rng(5)
    for _ in range(20):
        S = rng.choice(300, size=int(rng.integers(1, 12)), replace=False)
        a = oracle.f_alg1(V, S)
        b = oracle.f(V, S)
        assert a == pytest.approx(b, rel=1e-12, abs=1e-13)


def test_duplicate_members_do_not_change_f():
    V = _rand(50, 4, 3)
    assert oracle.f(V, [3, 7, 3, 7, 7]) == oracle.f(V, [3, 7])


def test_library_route_cdist():
    torch = pytest.importorskip("torch")
    V = _rand(400, 9, 4)
    Vd = torch.from_numpy(V.astype(np.float64))
    rng = np.random.default_rng(6)
    for _ in range(10):
        S = rng.choice(400, size=int(rng.integers(1, 20)), replace=False)
        ex = torch.cat([torch.zeros(1, 9, dtype=torch.float64), Vd[torch.from_numpy(S)]], 0)
        dmin = torch.cdist(Vd, ex).pow(2).min(dim=1).values.mean().item()
        l0 = Vd.pow(2).sum(1).mean().item()
        assert oracle.loss(V, S, with_e0=True) == pytest.approx(dmin, rel=1e-9)
        assert oracle.f(V, S) == pytest.approx(l0 - dmin, rel=1e-8, abs=1e-10)


def _all_subsets(n):
    for r in range(n + 1):
        for S in itertools.combinations(range(n), r):
            yield S


def test_monotone_and_submodular_exhaustive():
    # Def. 3 (monotone) and Def. 2 (diminishing returns) over every pair
    # A subset of B of a 7-point ground set.
    V = _rand(7, 3, 7)
    n = V.shape[0]
    fv = {S: oracle.f(V, list(S)) for S in _all_subsets(n)}
    for A in fv:
        for e in range(n):
            if e in A:
                continue
            Ae = tuple(sorted(A + (e,)))
            dA = fv[Ae] - fv[A]
            assert dA >= -1e-12  # monotone
            # every superset B of A not containing e
            rest = [x for x in range(n) if x not in A and x != e]
            for r in range(len(rest) + 1):
                for extra in itertools.combinations(rest, r):
                    B = tuple(sorted(A + extra))
                    Be = tuple(sorted(B + (e,)))
                    assert dA >= fv[Be] - fv[B] - 1e-12


def test_gains_are_discrete_derivatives():
    # Def. 1: Delta_f(c|S) = f(S u {c}) - f(S); oracle.gains works from the
    # per-point minima, oracle.f from the set directly.
    V = _rand(120, 6, 8)
    S = [5, 17, 60]
    m = oracle.norms(V)
    for s in S:
        oracle.update_m(V, m, s)
    cand = np.arange(120, dtype=np.int32)
    g = oracle.gains(V, m, cand)
    fS = oracle.f(V, S)
    for c in [0, 5, 33, 90, 119]:
        ref = oracle.f(V, S + [c]) - fS
        assert g[c] == pytest.approx(ref, rel=1e-10, abs=1e-12)
    # already-selected candidates gain exactly nothing
    assert g[5] == 0.0 and g[17] == 0.0 and g[60] == 0.0
    # gains are non-negative
    assert (g >= 0).all()


def test_greedy_telescopes_and_matches_direct_f():
    V = _rand(200, 5, 9)
    idx, fv, gap = oracle.greedy(V, 8)
    assert len(set(idx.tolist())) == 8
    for t in range(8):
        S = idx[: t + 1]
        assert fv[t] == pytest.approx(oracle.f(V, S), rel=1e-12)
        assert fv[t] == pytest.approx(oracle.f_alg1(V, S), rel=1e-11)
    assert np.all(np.diff(fv) >= 0)
    assert np.all((gap >= 0) & (gap <= 1))


def test_greedy_step_is_argmax_brute_force():
    # each pick maximises f(S u {c}) over every unselected c (Sec. 4.1)
    V = _rand(30, 4, 10)
    idx, fv, _ = oracle.greedy(V, 5)
    S = []
    for t in range(5):
        vals = [(oracle.f(V, S + [c]), -c) for c in range(30) if c not in S]
        best = max(vals)
        assert idx[t] == -best[1]
        S.append(int(idx[t]))


def test_greedy_resume_equals_one_shot():
    V = _rand(80, 3, 11)
    i1, f1, _ = oracle.greedy(V, 6)
    m = oracle.norms(V)
    sel = np.zeros(80, np.uint8)
    a, fa, _ = oracle.greedy(V, 3, m=m, selected=sel)
    b, fb, _ = oracle.greedy(V, 3, m=m, selected=sel, f_start=fa[-1])
    assert np.concatenate([a, b]).tolist() == i1.tolist()
    np.testing.assert_allclose(np.concatenate([fa, fb]), f1, rtol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_greedy_one_minus_inv_e_bound(seed):
    # Sec. 3: Greedy reaches at least (1 - 1/e) of the optimum
    V = _rand(12, 3, 100 + seed)
    for k in (1, 2, 3, 4):
        opt, _ = oracle.exhaustive_opt(V, k)
        _, fv, _ = oracle.greedy(V, k)
        assert fv[-1] >= (1 - 1 / math.e) * opt - 1e-12
        assert fv[-1] <= opt + 1e-12
    # k = 1: greedy is exact
    opt1, S1 = oracle.exhaustive_opt(V, 1)
    i1, f1, _ = oracle.greedy(V, 1)
    assert f1[0] == pytest.approx(opt1, rel=1e-15)


def test_errors():
    V = _rand(10, 2, 12)
    with pytest.raises(oracle.OracleError):
        oracle.f(V, [10])
    with pytest.raises(oracle.OracleError):
        oracle.f(V, [-1])
    with pytest.raises(oracle.OracleError):
        oracle.greedy(V, 11)
    with pytest.raises(oracle.OracleError):
        oracle.eval_sets(V, np.array([0, 1], np.int32), np.array([0, 2, 1], np.int64))
    # empty set list and empty sets
    assert oracle.eval_sets(V, np.zeros(0, np.int32), np.zeros(1, np.int64)).size == 0
    np.testing.assert_array_equal(
        oracle.eval_sets(V, np.array([3], np.int32), np.array([0, 0, 1, 1], np.int64))[[0, 2]], [0.0, 0.0])


def test_thread_count_does_not_change_results():
    V = _rand(500, 8, 13)
    m = oracle.norms(V)
    cand = np.arange(500, dtype=np.int32)
    a = oracle.gains(V, m, cand, threads=1)
    b = oracle.gains(V, m, cand, threads=4)
    np.testing.assert_array_equal(a, b)
