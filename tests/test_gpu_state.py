"""Greedy state snapshots (ebc_state_save / ebc_state_load): a Greedy
resumed from a snapshot, in the same or another handle over the same V,
continues with bitwise the picks and f of an uninterrupted run, and with the
picks and f of the FP64 oracle continued from the same state (S, m_v, f)."""
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


def gmm(n, d, seed):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, 7, sigma=None))


@pytest.mark.parametrize("prec,lazy", [("fp32", False), ("bf16", False), ("bf16", True), ("fp8", False)])
def test_resume_equals_uninterrupted(torch, prec, lazy):
    V = gmm(6000, 48, 21)
    with ebc.Instance(V, precision=prec, lazy=lazy) as a:
        ia, fa = a.greedy_host(12)
        st_a = a.stats()
    with ebc.Instance(V, precision=prec, lazy=lazy) as b:
        ib1, fb1 = b.greedy_host(5)
        snap = b.save_state()
        ib2, fb2 = b.greedy_host(7)
        b.reset()
        b.load_state(snap)  # same handle, after a reset
        ib3, fb3 = b.greedy_host(7)
    with ebc.Instance(V, precision=prec, lazy=lazy) as c:
        c.load_state(snap)  # another handle over the same V
        ic, fc = c.greedy_host(7)
        assert abs(c.current_f() - fa[-1]) <= 1e-9 * fa[-1]
        st_c = c.stats()
    for idx, f in ((ib2, fb2), (ib3, fb3), (ic, fc)):
        np.testing.assert_array_equal(np.concatenate([ib1, idx]), ia)
        np.testing.assert_array_equal(np.concatenate([fb1, f]), fa)
    assert st_c["rounds"] == st_a["rounds"] == 12


def _oracle_continue(V, picks, k):
    """The oracle's Greedy continued for k rounds from the state the picks
    reach (m_v updated by the oracle's own distances, f its own f(S))."""
    m = oracle.norms(V)
    sel = np.zeros(V.shape[0], dtype=np.uint8)
    for c in picks:
        oracle.update_m(V, m, int(c))
        sel[int(c)] = 1
    return oracle.greedy(V, k, m=m, selected=sel, f_start=oracle.f(V, picks))


@pytest.mark.parametrize("prec,lazy", [("fp32", False), ("bf16", False), ("bf16", True), ("fp16", False),
                                       ("fp8", False)])
def test_resume_matches_oracle(torch, prec, lazy):
    V = gmm(5000, 24, 33)
    with ebc.Instance(V, precision=prec, lazy=lazy) as b:
        i1, f1 = b.greedy_host(6)
        snap = b.save_state()
    ref_i, ref_f, ref_gap = _oracle_continue(V, i1, 9)
    with ebc.Instance(V, precision=prec, lazy=lazy) as c:
        c.load_state(snap)
        assert abs(c.current_f() - oracle.f(V, i1)) <= 1e-5 * oracle.f(V, i1)
        i2, f2 = c.greedy_host(9)
    for t in range(9):
        if ref_gap[t] > 1e-6:
            assert i2[t] == ref_i[t], (prec, t, i2.tolist(), ref_i.tolist())
        if i2[t] != ref_i[t]:
            break  # a legal divergence at a near-tie: compare f from here on
    np.testing.assert_allclose(f2, ref_f, rtol=1e-5)
    np.testing.assert_allclose(f2[-1], oracle.f(V, np.concatenate([i1, i2])), rtol=1e-5)


def test_state_errors(torch):
    V = gmm(500, 8, 3)
    with ebc.Instance(V) as a, ebc.Instance(gmm(400, 8, 4)) as b:
        a.greedy_host(3)
        snap = a.save_state()
        with pytest.raises(ebc.EbcError) as ei:
            b.load_state(snap)  # another shape
        assert ei.value.status == ebc.EBC_EINVAL
        with pytest.raises(ebc.EbcError):
            a.load_state(snap[: len(snap) // 2])  # truncated
        bad = bytearray(snap)
        bad[0] ^= 0xFF
        with pytest.raises(ebc.EbcError):
            a.load_state(bytes(bad))  # not a snapshot
        flags = bytearray(snap)
        flags[-1] ^= 1  # a selection flag that disagrees with the header
        with pytest.raises(ebc.EbcError):
            a.load_state(bytes(flags))
        a.load_state(snap)  # the handle is still usable
        a.greedy_host(2)
