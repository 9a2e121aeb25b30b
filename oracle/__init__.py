"""CPU oracle for exemplar-based clustering (FP64, plain C).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline / reference leg.  The GPU library never imports,
links or calls anything here, and nothing here calls the GPU library.

Functions (see ebc_oracle.c for the definitions and the paper sections each
one follows):

- ``sqdist(x, y)``              squared Euclidean distance, direct, FP64
- ``loss(V, S, with_e0)``       k-medoids loss L of Algorithm 1
- ``f_alg1(V, S)``              f(S) = L({e0}) - L(S u {e0})     (form A)
- ``f(V, S)``                   f(S) = mean_v max(0, |v|^2 - min_s d(v,s))  (form B)
- ``eval_sets(V, idx, off)``    form B for every set of a CSR list
- ``norms(V)``                  |v|^2 (distance to e0)
- ``gains(V, m, cand)``         mean_v max(0, m_v - d(v, c)) per candidate
- ``update_m(V, m, c)``         m_v <- min(m_v, d(v, c)) in place
- ``greedy(V, k, ...)``         Greedy with smallest-index tie-break
- ``exhaustive_opt(V, k)``      max over |S| = k of f(S), n <= 24
- ``sieve(V, items, K, thr, patience, ...)``  threshold sieve over a stream
- ``threshold_ladder(m, K, eps, upper)``  {(1+eps)^i : m <= (1+eps)^i <= upper K m}
- ``three_sieves(V, items, K, eps, T, m)`` / ``sieve_streaming(V, items, K, eps, m)``

Parity unpinned: none.  Every function is pinned by tests that do not call
it to produce its own expectation (closed forms, hand-computed fixtures in
tests/golden/, brute force, invariants, a library cross-check).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libebc_oracle.so")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_sqdist.restype = ctypes.c_double
            lib.orc_sqdist.argtypes = [_P, _P, _I32]
            lib.orc_loss.restype = ctypes.c_double
            lib.orc_loss.argtypes = [_P, _I64, _I32, _P, _I64, ctypes.c_int]
            for name in ("orc_f_alg1", "orc_f"):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [_P, _I64, _I32, _P, _I64, _P]
            lib.orc_eval_sets.restype = ctypes.c_int
            lib.orc_eval_sets.argtypes = [_P, _I64, _I32, _P, _P, _I64, _P, ctypes.c_int]
            lib.orc_norms.restype = None
            lib.orc_norms.argtypes = [_P, _I64, _I32, _P]
            lib.orc_gains.restype = ctypes.c_int
            lib.orc_gains.argtypes = [_P, _I64, _I32, _P, _P, _I64, _P, ctypes.c_int]
            lib.orc_update_m.restype = ctypes.c_int
            lib.orc_update_m.argtypes = [_P, _I64, _I32, _P, _I32]
            lib.orc_greedy.restype = ctypes.c_int
            lib.orc_greedy.argtypes = [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P, ctypes.c_double,
                                       ctypes.c_int]
            lib.orc_exhaustive_opt.restype = ctypes.c_int
            lib.orc_exhaustive_opt.argtypes = [_P, _I64, _I32, _I32, _P, _P]
            lib.orc_sieve.restype = ctypes.c_int
            lib.orc_sieve.argtypes = [_P, _I64, _I32, _P, _I64, _I32, _P, _I32, _I64, _P, _P, _P, _P, _P, _P,
                                      _P, _P, _P]
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError({-1: "EINVAL", -2: "EINDEX", -3: "ENOMEM"}.get(rc, str(rc)))


def _f32(V):
    V = np.ascontiguousarray(V, dtype=np.float32)
    if V.ndim != 2:
        raise ValueError("V must be 2-D (n, d)")
    return V


def _ptr(a):
    return a.ctypes.data_as(_P)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def sqdist(x, y) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    assert x.size == y.size
    return float(_load().orc_sqdist(_ptr(x), _ptr(y), x.size))


def loss(V, S, with_e0: bool = True) -> float:
    V = _f32(V)
    S = np.ascontiguousarray(S, dtype=np.int32).ravel()
    return float(_load().orc_loss(_ptr(V), V.shape[0], V.shape[1], _ptr(S), S.size, int(with_e0)))


def f_alg1(V, S) -> float:
    V = _f32(V)
    S = np.ascontiguousarray(S, dtype=np.int32).ravel()
    out = ctypes.c_double()
    _check(_load().orc_f_alg1(_ptr(V), V.shape[0], V.shape[1], _ptr(S), S.size, ctypes.byref(out)))
    return out.value


def f(V, S) -> float:
    V = _f32(V)
    S = np.ascontiguousarray(S, dtype=np.int32).ravel()
    out = ctypes.c_double()
    _check(_load().orc_f(_ptr(V), V.shape[0], V.shape[1], _ptr(S), S.size, ctypes.byref(out)))
    return out.value


def eval_sets(V, idx, off, threads: int = 0) -> np.ndarray:
    V = _f32(V)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    l = off.size - 1
    out = np.zeros(max(l, 0), dtype=np.float64)
    _check(_load().orc_eval_sets(_ptr(V), V.shape[0], V.shape[1], _ptr(idx), _ptr(off), l,
                                 _ptr(out), threads))
    return out


def norms(V) -> np.ndarray:
    V = _f32(V)
    out = np.zeros(V.shape[0], dtype=np.float64)
    _load().orc_norms(_ptr(V), V.shape[0], V.shape[1], _ptr(out))
    return out


def gains(V, m, cand, threads: int = 0) -> np.ndarray:
    V = _f32(V)
    m = np.ascontiguousarray(m, dtype=np.float64)
    cand = np.ascontiguousarray(cand, dtype=np.int32).ravel()
    assert m.size == V.shape[0]
    out = np.zeros(cand.size, dtype=np.float64)
    _check(_load().orc_gains(_ptr(V), V.shape[0], V.shape[1], _ptr(m), _ptr(cand), cand.size,
                             _ptr(out), threads))
    return out


def update_m(V, m, c) -> None:
    V = _f32(V)
    assert m.dtype == np.float64 and m.flags.c_contiguous and m.size == V.shape[0]
    _check(_load().orc_update_m(_ptr(V), V.shape[0], V.shape[1], _ptr(m), int(c)))


def greedy(V, k: int, m=None, selected=None, f_start: float = 0.0, threads: int = 0):
    """Greedy; returns (idx int32[k], f float64[k], gap float64[k]).

    ``m`` / ``selected`` (float64[n] / uint8[n]) continue from a state and are
    updated in place; leave both None to start from S = {}.
    """
    V = _f32(V)
    idx = np.full(k, -1, dtype=np.int32)
    fv = np.zeros(k, dtype=np.float64)
    gap = np.zeros(k, dtype=np.float64)
    mp = _ptr(m) if m is not None else None
    sp = _ptr(selected) if selected is not None else None
    if m is not None:
        assert m.dtype == np.float64 and m.flags.c_contiguous
        assert selected.dtype == np.uint8 and selected.flags.c_contiguous
    _check(_load().orc_greedy(_ptr(V), V.shape[0], V.shape[1], int(k), _ptr(idx), _ptr(fv), _ptr(gap),
                              mp, sp, float(f_start), threads))
    return idx, fv, gap


def exhaustive_opt(V, k: int):
    V = _f32(V)
    out = ctypes.c_double()
    S = np.zeros(max(k, 1), dtype=np.int32)
    _check(_load().orc_exhaustive_opt(_ptr(V), V.shape[0], V.shape[1], int(k), ctypes.byref(out), _ptr(S)))
    return out.value, S[:k].copy()


def sieve(V, items, K: int, thresholds, patience: int, m=None, selected=None, f_start: float = 0.0,
          level: int = 0, rejections: int = 0):
    """Threshold sieve over the stream ``items`` (see orc_sieve).

    Returns a dict with ``idx`` / ``f`` (accepted items, f after each),
    ``margin`` (per decided stream position), ``level``, ``rejections``
    and ``f_end``.  ``m`` / ``selected`` continue from a state and are updated
    in place (both None: S = {}).
    """
    V = _f32(V)
    n = V.shape[0]
    items = np.ascontiguousarray(items, dtype=np.int32).ravel()
    thr = np.ascontiguousarray(thresholds, dtype=np.float64).ravel()
    if m is None:
        m = norms(V)
        selected = np.zeros(n, dtype=np.uint8)
    assert m.dtype == np.float64 and m.flags.c_contiguous and m.size == n
    assert selected.dtype == np.uint8 and selected.flags.c_contiguous and selected.size == n
    idx = np.full(max(K, 1), -1, dtype=np.int32)
    fv = np.zeros(max(K, 1), dtype=np.float64)
    margin = np.full(max(items.size, 1), np.nan, dtype=np.float64)
    f_io = ctypes.c_double(f_start)
    lev = ctypes.c_int32(level)
    rej = ctypes.c_int64(rejections)
    cnt = ctypes.c_int32(0)
    _check(_load().orc_sieve(_ptr(V), n, V.shape[1], _ptr(items), items.size, int(K), _ptr(thr), thr.size,
                             int(patience), _ptr(m), _ptr(selected), ctypes.byref(f_io), ctypes.byref(lev),
                             ctypes.byref(rej), _ptr(idx), _ptr(fv), _ptr(margin), ctypes.byref(cnt)))
    c = cnt.value
    return {"idx": idx[:c].copy(), "f": fv[:c].copy(), "margin": margin[:items.size].copy(),
            "level": lev.value, "rejections": rej.value, "f_end": f_io.value}


def threshold_ladder(m_single: float, K: int, eps: float, upper: float = 1.0) -> np.ndarray:
    """Thresholds {(1+eps)^i : i integer, m <= (1+eps)^i <= upper K m}, largest first.

    The candidate values of OPT that Sieve Streaming (upper = 2) and Three
    Sieves (upper = 1) walk; each value is (1+eps)**i in double.
    """
    if not (m_single > 0.0 and eps > 0.0 and K >= 1 and upper > 0.0):
        raise ValueError("threshold_ladder needs m > 0, eps > 0, K >= 1, upper > 0")
    base = 1.0 + eps
    hi = upper * K * m_single
    i = math.floor(math.log(m_single) / math.log(base)) - 2
    while base ** i < m_single:
        i += 1
    out = []
    while base ** i <= hi:
        out.append(base ** i)
        i += 1
    return np.array(out[::-1], dtype=np.float64)


def three_sieves(V, items, K: int, eps: float, T: int, m_single: float):
    """Three Sieves: one summary, thresholds from K m down to m, moving down
    after T consecutive rejections."""
    return sieve(V, items, K, threshold_ladder(m_single, K, eps, 1.0), T)


def sieve_streaming(V, items, K: int, eps: float, m_single: float):
    """Sieve Streaming with a known largest singleton value m: one sieve per
    threshold of the ladder up to 2 K m; returns (best sieve's result,
    all results, thresholds)."""
    thr = threshold_ladder(m_single, K, eps, 2.0)
    res = [sieve(V, items, K, [v], 0) for v in thr]
    best = max(range(len(res)), key=lambda j: (res[j]["f_end"], -j))
    return res[best], res, thr
