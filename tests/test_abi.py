"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/ebc.h declares, and rejects bad arguments on the host before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2105_12026_gb300 import build as _build
from paper_2105_12026_gb300 import ebc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ebc.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ebc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ebc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_calls():
    names = declared_functions()
    for required in ("ebc_create", "ebc_eval_sets", "ebc_gains", "ebc_greedy", "ebc_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_every_symbol():
    assert set(declared_functions()) <= set(ebc._SIGS)


def test_version(lib):
    assert ebc.ebc_version() >= 1


@pytest.mark.parametrize("n,d", [(0, 4), (-5, 4), (10, 0), (10, 4097)])
def test_create_rejects_bad_sizes_on_host(lib, n, d):
    V = np.zeros((max(n, 1), max(d, 1)), np.float32)
    with pytest.raises(ebc.EbcError) as ei:
        ebc.ebc_create(V.ctypes.data, n, d, False, stream=0)
    assert ei.value.status == ebc.EBC_EINVAL


def test_create_rejects_null(lib):
    with pytest.raises(ebc.EbcError) as ei:
        ebc.ebc_create(0, 10, 4, False, stream=0)
    assert ei.value.status == ebc.EBC_EINVAL
    assert "NULL" in ebc.ebc_last_error(None)


def test_null_handle_calls_are_rejected(lib):
    assert lib.ebc_reset(None) == ebc.EBC_EINVAL
    assert lib.ebc_sync(None) == ebc.EBC_EINVAL
    assert lib.ebc_destroy(None) == ebc.EBC_OK


def test_no_gpu_gives_enodev_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    V = np.zeros((4, 2), np.float32)
    with pytest.raises(ebc.EbcError) as ei:
        ebc.ebc_create(V.ctypes.data, 4, 2, False, stream=0)
    assert ei.value.status == ebc.EBC_ENODEV


def test_estimate_bytes(lib):
    a = ebc.ebc_estimate_bytes(1000, 16, ebc.EBC_FP32)
    b = ebc.ebc_estimate_bytes(100000, 16, ebc.EBC_FP32)
    c = ebc.ebc_estimate_bytes(100000, 16, ebc.EBC_BF16)
    assert 0 < a < b < c
    assert ebc.ebc_estimate_bytes(0, 16, 0) == -1


def test_batch_create_rejects_bad_arguments(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.ebc_batch_create(0, 1 << 30, 8, ctypes.byref(h)) == ebc.EBC_EINVAL
    assert lib.ebc_batch_create(4, 0, 8, ctypes.byref(h)) == ebc.EBC_EINVAL
    assert lib.ebc_batch_create(4, 1 << 30, 0, ctypes.byref(h)) == ebc.EBC_EINVAL
    assert lib.ebc_batch_submit(None, None, 10, 4, 2, 0, None) == ebc.EBC_EINVAL


def test_tune_table_json_roundtrip(lib, tmp_path):
    """The tuning table persists as JSON; malformed files are rejected and
    leave the table unchanged (no GPU needed)."""
    ebc.ebc_tune_clear()
    assert ebc.ebc_tune_count() == 0
    good = tmp_path / "tune.json"
    good.write_text('{"version": 1, "entries": [\n'
                    ' {"prec": 1, "rb": 256, "nbucket": 17, "na": 1, "ns": 2, "chunk": 0, "ms": 7.2},\n'
                    ' {"ns": 3, "na": 2, "prec": 3, "rb": 128, "nbucket": 12, "chunk": 1, "bn": 128}\n]}\n')
    ebc.ebc_tune_load(str(good))
    assert ebc.ebc_tune_count() == 2
    out = tmp_path / "out.json"
    ebc.ebc_tune_save(str(out))
    ebc.ebc_tune_clear()
    ebc.ebc_tune_load(str(out))
    assert ebc.ebc_tune_count() == 2
    text = out.read_text()
    assert '"rb": 256' in text and '"chunk": 1' in text
    assert text.count('"bn": 128') == 1 and text.count('"bn": 256') == 1  # absent width: 256
    assert text.count('"turns": -1') == 2  # absent: by row width
    assert text.count('"es": 0') == 2  # absent: column halves
    for bad in ['{"entries": [{"prec": 1, "rb": 256}]}',
                '{"entries": [{"prec": 9, "rb": 256, "nbucket": 3, "na": 1, "ns": 2, "chunk": 0}]}',
                '{"entries": [{"prec": 1, "rb": 256, "nbucket": 3, "na": 1, "ns": 2, "chunk": 0, "bn": 64}]}',
                '{"entries": [{"prec": 1, "rb": 256, "nbucket": 3, "na": 1, "ns": 2, "chunk": 0, "turns": 2}]}',
                '{"entries": [{"prec": 1, "rb": 256, "nbucket": 3, "na": 1, "ns": 2, "chunk": 0, "bn": 128, "es": 1}]}',
                'not json']:
        p = tmp_path / "bad.json"
        p.write_text(bad)
        with pytest.raises(ebc.EbcError) as ei:
            ebc.ebc_tune_load(str(p))
        assert ei.value.status == ebc.EBC_EINVAL
    assert ebc.ebc_tune_count() == 2
    with pytest.raises(ebc.EbcError):
        ebc.ebc_tune_load(str(tmp_path / "missing.json"))
    ebc.ebc_tune_clear()


@pytest.mark.parametrize("m,K,eps,upper", [(0.5553, 5, 0.2, 1.0), (1.0, 10, 0.1, 2.0), (3.7e-3, 100, 0.01, 1.0),
                                           (1.0, 1, 1.0, 1.0), (7.0, 3, 0.5, 2.0), (18.34, 100, 0.001, 1.0),
                                           (1e-30, 7, 0.3, 2.0), (2.0 ** 40, 50, 0.05, 1.0)])
def test_threshold_ladder_matches_oracle(lib, m, K, eps, upper):
    """The library's ladder (host logic of the streaming optimisers) equals
    the oracle's, value for value."""
    import oracle
    got = ebc.ebc_threshold_ladder(m, K, eps, upper)
    ref = oracle.threshold_ladder(m, K, eps, upper)
    np.testing.assert_array_equal(got, ref)
    assert got.size >= 1 and np.all(np.diff(got) < 0)


def test_threshold_ladder_errors(lib):
    cnt = ctypes.c_int32()
    f = lib.ebc_threshold_ladder
    for args in [(0.0, 5, 0.1, 1.0), (1.0, 0, 0.1, 1.0), (1.0, 5, 0.0, 1.0), (1.0, 5, 0.1, 0.0),
                 (float("inf"), 5, 0.1, 1.0), (float("nan"), 5, 0.1, 1.0), (1.0, 5, 1e-12, 1.0)]:
        assert f(*args, None, 0, ctypes.byref(cnt)) == ebc.EBC_EINVAL, args
    assert f(1.0, 5, 0.1, 1.0, None, 0, None) == ebc.EBC_EINVAL
    assert f(1.0, 4, 1.0, 1.0, None, 0, ctypes.byref(cnt)) == ebc.EBC_OK and cnt.value == 3  # 4, 2, 1
    out = np.zeros(2)
    assert f(1.0, 4, 1.0, 1.0, out.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(cnt)) == ebc.EBC_EINVAL


def test_sieve_rejects_null_handle(lib):
    st = ebc.ebc_sieve_state()
    cnt = ctypes.c_int32()
    assert lib.ebc_sieve_host(None, ctypes.byref(st), None, 0, None, None, ctypes.byref(cnt)) == ebc.EBC_EINVAL
    assert lib.ebc_gain_bounds(None, None, 0, None) == ebc.EBC_EINVAL
    assert lib.ebc_set_kblocked(None, 1) == ebc.EBC_EINVAL
