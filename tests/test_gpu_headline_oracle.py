"""The headline Greedy configuration against the FP64 oracle, round by round.

Drifting-regime features, n = 200,000, d = 128, k = 100, BF16 tensor cores
with certified picks (Sec. 3 Greedy; the step of Sec. 4.1).  The oracle
cannot run Greedy itself at this size (4e10 distances per round), so it
follows the GPU's picks and checks each one:

* f grows by the oracle's exact gain of the pick (1e-5 relative);
* no candidate in a seeded sample of 512 unselected points, nor any
  candidate of the round's certified stage (top list and escalation list),
  has a larger oracle gain than the pick (beyond the 1e-10 tie margin);
* where the oracle's top-two gap over that pool exceeds 1e-6, the pick is
  the pool's argmax;
* the final f equals the oracle's f(S) of the picks (1e-5 relative).

At this size the bulk kernel splits V into many chunks, almost every round
escalates (tens to hundreds of candidates), and the lazy and FP8 Greedy run
in lockstep and must make the same picks.
"""
import numpy as np
import pytest

import oracle
from paper_2105_12026_gb300 import ebc, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2105_12026_gb300 import build
    build.build()
    ebc.load()
    t.cuda.set_device(0)
    return t


def test_headline_greedy_rounds_against_oracle(torch):
    w = synth.regime_greedy(seed=0)
    V, k = w["V"], w["k"]
    n = V.shape[0]
    rng = np.random.default_rng(2024)
    m = oracle.norms(V)
    sel = np.zeros(n, dtype=np.uint8)
    Vd = torch.from_numpy(V).cuda()
    picks, f_prev, escalated = [], 0.0, 0
    with ebc.Instance(Vd, precision="bf16") as full, ebc.Instance(Vd, precision="bf16", lazy=True) as lazy, \
            ebc.Instance(Vd, precision="fp8") as fp8:
        for t in range(k):
            idx, fv = full.greedy_host(1)
            c = int(idx[0])
            stage = full.last_round_candidates()
            escalated += stage.size > full.stats()["refine_k"]
            li, lf = lazy.greedy_host(1)
            qi, qf = fp8.greedy_host(1)
            assert int(li[0]) == c and lf[0] == fv[0], (t, c, int(li[0]))
            assert int(qi[0]) == c and qf[0] == fv[0], (t, c, int(qi[0]))
            unsel = np.flatnonzero(sel == 0)
            sample = rng.choice(unsel, 512, replace=False)
            pool = np.unique(np.concatenate([sample, stage, [c]])).astype(np.int32)
            pool = pool[sel[pool] == 0]
            g = oracle.gains(V, m, pool)
            gc = float(g[pool == c][0])
            assert abs((fv[0] - f_prev) - gc) <= 1e-5 * gc, (t, fv[0] - f_prev, gc)
            assert g.max() <= gc * (1 + 1e-9), (t, c, int(pool[np.argmax(g)]), g.max(), gc)
            order = np.argsort(-g, kind="stable")
            if order.size > 1 and (g[order[0]] - g[order[1]]) > 1e-6 * g[order[0]]:
                assert int(pool[order[0]]) == c, (t, c, int(pool[order[0]]))
            f_prev = float(fv[0])
            oracle.update_m(V, m, c)
            sel[c] = 1
            picks.append(c)
    assert escalated >= 50  # the long escalation lists were exercised
    np.testing.assert_allclose(f_prev, oracle.f(V, np.array(picks, dtype=np.int32)), rtol=1e-5)
