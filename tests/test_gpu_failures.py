"""Failure paths, exercised without faulting the GPU.

* A bounded device wait that runs out: the limit of the tensor-core
  pipeline's waits is set to 1 ns, so waits on TMA copies, MMAs and the
  epilogue give up; each CTA records EBC_ETIMEOUT, waits (with the default
  limit) for the work it already issued, frees its tensor memory and
  returns.  Covered for the resident, K-blocked, 128-point-tile, FP8,
  multi-set and shared group kernels.  The host reads the status; with the default limit restored the
  same handle gives the same results as before, bitwise.
* A device allocation that fails (injected on the host, in the library's
  pool allocator): ebc_create and ebc_set_precision return EBC_ENOMEM and
  leave nothing half-built behind; in the batch runtime the request whose
  admission failed finishes with EBC_ENOMEM and the others are unaffected.
"""
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


@pytest.fixture(autouse=True)
def _defaults():
    yield
    ebc.ebc_set_wait_limit_ns(0)
    ebc.ebc_inject_alloc_failure(-1)


def gmm(n, d, seed):
    return synth.zscore_to_f32(synth.gaussian_mixture(np.random.default_rng(seed), n, d, 9, sigma=None))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_wait_timeout_reported_and_handle_recovers(torch, prec):
    V = gmm(20_000, 64, 1)
    sets = synth.random_sets(np.random.default_rng(2), V.shape[0], 200, 1, 32)
    with ebc.Instance(V, precision=prec) as inst:
        ref_g = inst.gains_host()
        ref_s = inst.eval_sets_host(*sets)
        ebc.ebc_set_wait_limit_ns(1)
        with pytest.raises(ebc.EbcError) as ei:
            inst.gains_host()
        assert ei.value.status == ebc.EBC_ETIMEOUT and "wait" in str(ei.value)
        with pytest.raises(ebc.EbcError) as ei:
            inst.eval_sets_host(*sets)
        assert ei.value.status == ebc.EBC_ETIMEOUT
        with pytest.raises(ebc.EbcError) as ei:
            inst.greedy_host(2)
        assert ei.value.status == ebc.EBC_ETIMEOUT
        ebc.ebc_set_wait_limit_ns(0)
        inst.reset()  # the timed-out Greedy rounds left picks of no meaning; gains are relative to S
        np.testing.assert_array_equal(inst.gains_host(), ref_g)
        np.testing.assert_array_equal(inst.eval_sets_host(*sets), ref_s)
        idx, f = inst.greedy_host(6)
    ref_i, ref_f, ref_gap = oracle.greedy(V, 6)
    for t in range(6):
        if ref_gap[t] > 1e-6:
            assert idx[t] == ref_i[t], (t, idx.tolist(), ref_i.tolist())
        if idx[t] != ref_i[t]:
            break
    np.testing.assert_allclose(f, ref_f, rtol=1e-5)


@pytest.mark.parametrize("case", ["kblocked", "tile128", "group"])
def test_wait_timeout_other_kernels(torch, case, tmp_path):
    """The same for the K-blocked kernel (d > 128), the 128-point tile shape
    (forced through a tuning-table entry) and the shared group launch: every
    variant's waits give up, report EBC_ETIMEOUT and leave the handles
    usable."""
    import json
    import math
    d = 256 if case == "kblocked" else 64
    V = gmm(12_000, d, 7)
    ebc.ebc_tune_clear()
    if case == "tile128":
        ent = {"prec": ebc.PRECISIONS["bf16"], "rb": 128, "nbucket": int(math.floor(math.log2(V.shape[0]))),
               "na": 2, "ns": 3, "chunk": 0, "bn": 128}
        path = tmp_path / "t.json"
        path.write_text(json.dumps({"version": 1, "entries": [ent]}))
        ebc.ebc_tune_load(str(path))
    try:
        with ebc.Instance(V, precision="bf16") as inst:
            if case == "tile128":
                assert inst.tune_entry()["bn"] == 128
            ref_g = inst.gains_host()
            ref_i, ref_f = inst.greedy_host(4)
            inst.reset()
            ebc.ebc_set_wait_limit_ns(1)
            if case == "group":
                with ebc.Group() as g:
                    g.greedy([inst], [2])
                with pytest.raises(ebc.EbcError) as ei:
                    inst.sync()
            else:
                with pytest.raises(ebc.EbcError) as ei:
                    inst.gains_host()
            assert ei.value.status == ebc.EBC_ETIMEOUT
            ebc.ebc_set_wait_limit_ns(0)
            inst.reset()
            np.testing.assert_array_equal(inst.gains_host(), ref_g)
            idx, f = inst.greedy_host(4)
        np.testing.assert_array_equal(idx, ref_i)
        np.testing.assert_array_equal(f, ref_f)
    finally:
        ebc.ebc_tune_clear()


def test_wait_limit_arguments(torch):
    for bad in (-1, 61_000_000_000):
        with pytest.raises(ebc.EbcError) as ei:
            ebc.ebc_set_wait_limit_ns(bad)
        assert ei.value.status == ebc.EBC_EINVAL
    with pytest.raises(ebc.EbcError):
        ebc.ebc_inject_alloc_failure(-2)


def test_create_out_of_memory_is_clean(torch):
    V = gmm(30_000, 32, 3)
    torch.cuda.synchronize()
    ebc.ebc_release_cached_memory()
    free0 = torch.cuda.mem_get_info()[0]
    for after in (0, 1, 4, 9, 15, 21):  # the failure lands at different points of ebc_create
        ebc.ebc_inject_alloc_failure(after)
        with pytest.raises(ebc.EbcError) as ei:
            ebc.Instance(V)
        assert ei.value.status == ebc.EBC_ENOMEM, after
    torch.cuda.synchronize()
    ebc.ebc_release_cached_memory()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)  # nothing left allocated
    with ebc.Instance(V) as inst:  # disarmed: works
        i1, f1 = inst.greedy_host(3)
    ref_i, ref_f, _ = oracle.greedy(V, 3)
    np.testing.assert_allclose(f1, ref_f, rtol=1e-5)


# Failure points, in order: the 11 tensor-core buffers; for FP8 then (once
# those exist) its 16 buffers, then the two lazy-bound arrays.
FAIL_AT = {"bf16": (0, 3, 7, 10), "fp8": (0, 5, 11, 8, 16, 1)}


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_set_precision_out_of_memory_then_retry(torch, prec):
    V = gmm(8_000, 48, 4)
    with ebc.Instance(V) as inst:
        for after in FAIL_AT[prec]:
            ebc.ebc_inject_alloc_failure(after)
            with pytest.raises(ebc.EbcError) as ei:
                inst.set_precision(prec)
            assert ei.value.status == ebc.EBC_ENOMEM
            assert inst.stats()["prec"] == ebc.PRECISIONS["fp32"]  # unchanged
        ebc.ebc_inject_alloc_failure(-1)
        inst.set_precision(prec)
        idx, f = inst.greedy_host(5)
    with ebc.Instance(V, precision=prec) as ref:
        ridx, rf = ref.greedy_host(5)
    np.testing.assert_array_equal(idx, ridx)
    np.testing.assert_array_equal(f, rf)


def test_batch_admission_out_of_memory(torch):
    rng = np.random.default_rng(6)
    specs = [(gmm(int(n), 32, 10 + i), int(rng.integers(3, 8))) for i, n in enumerate((4000, 2500, 6000))]
    with ebc.Batch(max_slots=1, budget_bytes=8 << 30) as b:  # one slot: admissions one after another
        tickets = [b.submit(V, k, "bf16") for V, k in specs]
        ebc.ebc_inject_alloc_failure(5)  # inside the first request's admission
        b.run()
        with pytest.raises(ebc.EbcError) as ei:
            b.poll(tickets[0])
        assert ei.value.status == ebc.EBC_ENOMEM
        got = [b.poll(t) for t in tickets[1:]]
        st = b.stats()
    assert st["completed"] == 3 and st["active"] == 0 and st["queued"] == 0
    for (V, k), res in zip(specs[1:], got):
        assert res is not None
        with ebc.Instance(V, precision="bf16") as inst:
            ridx, rf = inst.greedy_host(k)
        np.testing.assert_array_equal(res[0], ridx)
        np.testing.assert_array_equal(res[1], rf)
