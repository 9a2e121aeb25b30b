"""Thin Python binding of the C ABI in include/ebc.h (argument marshalling only).

Function names match the C entry points.  Device pointers are taken from
torch CUDA tensors (``tensor.data_ptr()``); streams from
``torch.cuda.current_stream().cuda_stream``.  Every step of the computation
runs in the CUDA library: if ``_build/libebc.so`` is missing this module
raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

EBC_OK, EBC_EINVAL, EBC_EINDEX, EBC_ENOMEM, EBC_ECUDA, EBC_ETIMEOUT, EBC_EBUSY, EBC_ENODEV = 0, -1, -2, -3, -4, -5, -6, -7
EBC_FP32, EBC_BF16, EBC_FP16, EBC_FP8E4M3 = 0, 1, 2, 3
PRECISIONS = {"fp32": EBC_FP32, "bf16": EBC_BF16, "fp16": EBC_FP16, "fp8": EBC_FP8E4M3}
_NAMES = {EBC_EINVAL: "EINVAL", EBC_EINDEX: "EINDEX", EBC_ENOMEM: "ENOMEM", EBC_ECUDA: "ECUDA",
          EBC_ETIMEOUT: "ETIMEOUT", EBC_EBUSY: "EBUSY", EBC_ENODEV: "ENODEV"}


class EbcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class ebc_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("certified_rounds", ctypes.c_int64),
                ("escalated_rounds", ctypes.c_int64), ("escalated_candidates", ctypes.c_int64),
                ("max_raw_rel_err", ctypes.c_double), ("exact_evaluations", ctypes.c_int64),
                ("prec", ctypes.c_int32), ("refine_k", ctypes.c_int32), ("bulk_candidates", ctypes.c_int64),
                ("lazy", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ebc_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("bulk_launches", ctypes.c_int64), ("bulk_ms", ctypes.c_double),
                ("bulk_evals", ctypes.c_int64), ("refine_launches", ctypes.c_int64), ("refine_ms", ctypes.c_double),
                ("eval_launches", ctypes.c_int64), ("eval_ms", ctypes.c_double),
                ("list_launches", ctypes.c_int64), ("list_ms", ctypes.c_double)]


class ebc_batch_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64), ("bytes_peak", ctypes.c_int64),
                ("rounds_issued", ctypes.c_int64), ("evals_full", ctypes.c_int64),
                ("evals_performed", ctypes.c_int64)]


class ebc_sieve_state(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("nthr", ctypes.c_int32), ("thr", ctypes.c_void_p),
                ("patience", ctypes.c_int64), ("level", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rejections", ctypes.c_int64), ("consumed", ctypes.c_int64), ("bounded", ctypes.c_int64),
                ("exact", ctypes.c_int64), ("bounds", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

# name -> argtypes (restype is ebc_status = int unless noted)
_SIGS = {
    "ebc_version": [],
    "ebc_create": [_P, _I64, _I32, _I32, _P, ctypes.POINTER(_P)],
    "ebc_reload": [_P, _P, _I32],
    "ebc_destroy": [_P],
    "ebc_set_profiling": [_P, _I32],
    "ebc_get_profile": [_P, ctypes.POINTER(ebc_profile)],
    "ebc_reset_profile": [_P],
    "ebc_set_stream": [_P, _P],
    "ebc_set_precision": [_P, ctypes.c_int, _I32],
    "ebc_eval_sets": [_P, _P, _P, _I64, _P],
    "ebc_eval_sets_host": [_P, _P, _P, _I64, _P],
    "ebc_gains": [_P, _P, _I64, _P],
    "ebc_gains_host": [_P, _P, _I64, _P],
    "ebc_greedy": [_P, _I32, _P, _P],
    "ebc_greedy_host": [_P, _I32, _P, _P],
    "ebc_gain_bounds": [_P, _P, _I64, _P],
    "ebc_gain_bounds_host": [_P, _P, _I64, _P],
    "ebc_sieve_host": [_P, ctypes.POINTER(ebc_sieve_state), _P, _I64, _P, _P, ctypes.POINTER(_I32)],
    "ebc_threshold_ladder": [ctypes.c_double, _I32, ctypes.c_double, ctypes.c_double, _P, _I32,
                             ctypes.POINTER(_I32)],
    "ebc_set_graphs": [_P, _I32],
    "ebc_set_wait_limit_ns": [_I64],
    "ebc_inject_alloc_failure": [_I64],
    "ebc_set_kblocked": [_P, _I32],
    "ebc_set_lazy": [_P, _I32],
    "ebc_state_size": [_P, ctypes.POINTER(_I64)],
    "ebc_state_save": [_P, _P, _I64],
    "ebc_state_load": [_P, _P, _I64],
    "ebc_autotune": [_P, _I32],
    "ebc_tune_query": [_P, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)],
    "ebc_tune_save": [ctypes.c_char_p],
    "ebc_tune_load": [ctypes.c_char_p],
    "ebc_tune_count": [],
    "ebc_tune_clear": [],
    "ebc_batch_set_autotune": [_P, _I32],
    "ebc_set_max_ctas": [_P, _I32],
    "ebc_batch_set_large": [_P, _I64, _I32, _I32],
    "ebc_batch_set_lazy": [_P, _I32, _I64],
    "ebc_reset": [_P],
    "ebc_sync": [_P],
    "ebc_get_stats": [_P, ctypes.POINTER(ebc_stats)],
    "ebc_current_f": [_P, ctypes.POINTER(ctypes.c_double)],
    "ebc_reserve_sets": [_P, _I64, _I64],
    "ebc_last_round_candidates": [_P, _P, _I64, ctypes.POINTER(_I64)],
    "ebc_last_error": [_P],
    "ebc_eval_sets_noalloc": [_P, _I64, _I32, _P, _P, _I64, _P, _P],
    "ebc_noalloc_last_error": [],
    "ebc_estimate_bytes": [_I64, _I32, _I32],
    "ebc_release_cached_memory": [],
    "ebc_group_create": [ctypes.POINTER(_P)],
    "ebc_group_greedy": [_P, _P, _I32, _P, _P, _P],
    "ebc_group_stats": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "ebc_group_set_lanes": [_P, _I32],
    "ebc_group_set_lanes_by_row_width": [_P, _I32],
    "ebc_group_set_max_ctas": [_P, _I32],
    "ebc_group_set_profiling": [_P, _I32],
    "ebc_group_profile": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(_I64)],
    "ebc_group_reset_profile": [_P],
    "ebc_group_last_error": [_P],
    "ebc_group_destroy": [_P],
    "ebc_batch_create": [_I32, _I64, _I32, ctypes.POINTER(_P)],
    "ebc_batch_submit": [_P, _P, _I64, _I32, _I32, ctypes.c_int, ctypes.POINTER(_I64)],
    "ebc_batch_step": [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
    "ebc_batch_poll": [_P, _I64, _P, _P, _I32, ctypes.POINTER(_I32)],
    "ebc_batch_run": [_P],
    "ebc_batch_stats": [_P, ctypes.POINTER(ebc_batch_info)],
    "ebc_batch_last_error": [_P],
    "ebc_batch_destroy": [_P],
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the library (build it first with ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or library_path()
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
            lib = ctypes.CDLL(p)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.ebc_last_error.restype = ctypes.c_char_p
            lib.ebc_noalloc_last_error.restype = ctypes.c_char_p
            lib.ebc_batch_last_error.restype = ctypes.c_char_p
            lib.ebc_group_last_error.restype = ctypes.c_char_p
            lib.ebc_estimate_bytes.restype = ctypes.c_int64
            lib.ebc_tune_count.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _raise(h, rc):
    if rc != EBC_OK:
        msg = load().ebc_last_error(h)
        raise EbcError(rc, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------------------
# one wrapper per C entry point
# ---------------------------------------------------------------------------

def ebc_version() -> int:
    return int(load().ebc_version())


def ebc_create(V_ptr: int, n: int, d: int, v_on_device: bool, stream=None) -> int:
    h = _P()
    rc = load().ebc_create(_P(V_ptr), n, d, int(bool(v_on_device)), _P(_stream_ptr(stream)), ctypes.byref(h))
    _raise(None, rc)
    return h.value


def ebc_reload(h: int, V_ptr: int, v_on_device: bool) -> None:
    _raise(h, load().ebc_reload(_P(h), _P(V_ptr), int(bool(v_on_device))))


def ebc_set_profiling(h: int, on: bool) -> None:
    _raise(h, load().ebc_set_profiling(_P(h), int(bool(on))))


def ebc_get_profile(h: int) -> dict:
    p = ebc_profile()
    _raise(h, load().ebc_get_profile(_P(h), ctypes.byref(p)))
    return {k: getattr(p, k) for k, _ in ebc_profile._fields_}


def ebc_reset_profile(h: int) -> None:
    _raise(h, load().ebc_reset_profile(_P(h)))


def ebc_destroy(h: int) -> None:
    load().ebc_destroy(_P(h))


def ebc_set_stream(h: int, stream) -> None:
    _raise(h, load().ebc_set_stream(_P(h), _P(_stream_ptr(stream))))


def ebc_set_precision(h: int, prec: int, refine_k: int = 8) -> None:
    _raise(h, load().ebc_set_precision(_P(h), int(prec), int(refine_k)))


def ebc_eval_sets(h: int, idx_ptr: int, off_ptr: int, l: int, out_ptr: int) -> None:
    _raise(h, load().ebc_eval_sets(_P(h), _P(idx_ptr), _P(off_ptr), int(l), _P(out_ptr)))


def ebc_eval_sets_host(h: int, idx: np.ndarray, off: np.ndarray) -> np.ndarray:
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    l = off.size - 1
    out = np.zeros(max(l, 0), dtype=np.float64)
    _raise(h, load().ebc_eval_sets_host(_P(h), idx.ctypes.data_as(_P), off.ctypes.data_as(_P), l,
                                        out.ctypes.data_as(_P)))
    return out


def ebc_gains(h: int, cand_ptr, m: int, out_ptr: int) -> None:
    _raise(h, load().ebc_gains(_P(h), _P(cand_ptr), int(m), _P(out_ptr)))


def ebc_gains_host(h: int, cand: np.ndarray | None, m: int | None = None) -> np.ndarray:
    if cand is None:
        out = np.zeros(int(m), dtype=np.float64)
        _raise(h, load().ebc_gains_host(_P(h), None, int(m), out.ctypes.data_as(_P)))
        return out
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    out = np.zeros(cand.size, dtype=np.float64)
    _raise(h, load().ebc_gains_host(_P(h), cand.ctypes.data_as(_P), cand.size, out.ctypes.data_as(_P)))
    return out


def ebc_greedy(h: int, k: int, out_idx_ptr: int, out_f_ptr: int) -> None:
    _raise(h, load().ebc_greedy(_P(h), int(k), _P(out_idx_ptr), _P(out_f_ptr)))


def ebc_set_max_ctas(h: int, max_ctas: int) -> None:
    _raise(h, load().ebc_set_max_ctas(_P(h), int(max_ctas)))


def ebc_set_graphs(h: int, on: bool) -> None:
    _raise(h, load().ebc_set_graphs(_P(h), int(bool(on))))


def ebc_set_wait_limit_ns(ns: int) -> None:
    """Limit of each tensor-core pipeline wait (0: the default of 1 s)."""
    rc = load().ebc_set_wait_limit_ns(int(ns))
    if rc != EBC_OK:
        raise EbcError(rc, "ebc_set_wait_limit_ns: out of range")


def ebc_inject_alloc_failure(after: int) -> None:
    """Make the device allocation after `after` more successful ones fail (-1: disarm)."""
    rc = load().ebc_inject_alloc_failure(int(after))
    if rc != EBC_OK:
        raise EbcError(rc, "ebc_inject_alloc_failure: after < -1")


def ebc_autotune(h: int, reps: int = 3) -> None:
    _raise(h, load().ebc_autotune(_P(h), int(reps)))


def ebc_tune_save(path: str) -> None:
    _raise(None, load().ebc_tune_save(path.encode()))


def ebc_tune_load(path: str) -> None:
    _raise(None, load().ebc_tune_load(path.encode()))


def ebc_tune_count() -> int:
    return int(load().ebc_tune_count())


def ebc_tune_clear() -> None:
    _raise(None, load().ebc_tune_clear())


def ebc_set_lazy(h: int, on: bool) -> None:
    _raise(h, load().ebc_set_lazy(_P(h), int(bool(on))))


def ebc_greedy_host(h: int, k: int):
    idx = np.zeros(k, dtype=np.int32)
    f = np.zeros(k, dtype=np.float64)
    _raise(h, load().ebc_greedy_host(_P(h), int(k), idx.ctypes.data_as(_P), f.ctypes.data_as(_P)))
    return idx, f


def ebc_threshold_ladder(m: float, K: int, eps: float, upper: float = 1.0) -> np.ndarray:
    """Thresholds (1+eps)^i in [m, upper K m], largest first (host only)."""
    cnt = _I32()
    _raise(None, load().ebc_threshold_ladder(float(m), int(K), float(eps), float(upper), None, 0, ctypes.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), dtype=np.float64)
    _raise(None, load().ebc_threshold_ladder(float(m), int(K), float(eps), float(upper), out.ctypes.data_as(_P),
                                             cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def ebc_sieve_host(h: int, state: ebc_sieve_state, items: np.ndarray):
    """One pass of the threshold sieve over ``items``; returns the accepted
    (idx int32, f float64) and updates ``state`` in place."""
    items = np.ascontiguousarray(items, dtype=np.int32).ravel()
    room = max(int(state.K), 1)
    idx = np.zeros(room, dtype=np.int32)
    f = np.zeros(room, dtype=np.float64)
    cnt = _I32()
    _raise(h, load().ebc_sieve_host(_P(h), ctypes.byref(state), items.ctypes.data_as(_P), items.size,
                                    idx.ctypes.data_as(_P), f.ctypes.data_as(_P), ctypes.byref(cnt)))
    return idx[:cnt.value].copy(), f[:cnt.value].copy()


def ebc_reset(h: int) -> None:
    _raise(h, load().ebc_reset(_P(h)))


def ebc_sync(h: int) -> None:
    _raise(h, load().ebc_sync(_P(h)))


def ebc_get_stats(h: int) -> dict:
    s = ebc_stats()
    _raise(h, load().ebc_get_stats(_P(h), ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in ebc_stats._fields_}


def ebc_last_round_candidates(h: int) -> np.ndarray:
    """Candidates that reached the certified stage of the last Greedy round."""
    cnt = _I64()
    _raise(h, load().ebc_last_round_candidates(_P(h), None, 0, ctypes.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    _raise(h, load().ebc_last_round_candidates(_P(h), out.ctypes.data_as(_P), out.size, ctypes.byref(cnt)))
    return out[:cnt.value].copy()


def ebc_current_f(h: int) -> float:
    v = ctypes.c_double()
    _raise(h, load().ebc_current_f(_P(h), ctypes.byref(v)))
    return v.value


def ebc_eval_sets_noalloc(V_ptr: int, n: int, d: int, idx_ptr: int, off_ptr: int, l: int, out_ptr: int,
                          stream=None) -> None:
    """Allocation-free multi-set evaluation over device pointers (see include/ebc.h)."""
    rc = load().ebc_eval_sets_noalloc(_P(V_ptr), int(n), int(d), _P(idx_ptr), _P(off_ptr), int(l), _P(out_ptr),
                                      _P(_stream_ptr(stream)))
    if rc != EBC_OK:
        msg = load().ebc_noalloc_last_error()
        raise EbcError(rc, msg.decode() if msg else "")


def ebc_last_error(h: int | None) -> str:
    m = load().ebc_last_error(_P(h) if h else None)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# convenience object over torch tensors (marshalling only)
# ---------------------------------------------------------------------------

class Instance:
    """One resident ground set.  ``V`` is an (n, d) float32 torch tensor or numpy array."""

    def __init__(self, V, precision: str = "fp32", refine_k: int = 8, stream=None, lazy: bool = False):
        import torch
        self._keep = None
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float32)
            self.n, self.d = V.shape
            self.h = ebc_create(V.ctypes.data, self.n, self.d, False, stream)
        else:
            if V.dtype != torch.float32 or V.dim() != 2:
                raise ValueError("V must be a 2-D float32 tensor")
            V = V.contiguous()
            self.n, self.d = V.shape
            self.h = ebc_create(V.data_ptr(), self.n, self.d, V.is_cuda, stream)
        self.precision = precision
        if precision != "fp32" or refine_k != 8:
            ebc_set_precision(self.h, PRECISIONS[precision], refine_k)
        if lazy:
            ebc_set_lazy(self.h, True)

    def close(self):
        if getattr(self, "h", None):
            ebc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_lazy(self, on: bool = True):
        ebc_set_lazy(self.h, on)

    def set_kblocked(self, on: bool = True):
        _raise(self.h, load().ebc_set_kblocked(_P(self.h), int(bool(on))))

    def autotune(self, reps: int = 3):
        ebc_autotune(self.h, reps)

    def tune_entry(self):
        """The tuning-table entry bulk launches of this instance use at its
        current precision: dict(bn, na, ns, chunk, turns, es, ms), or None when
        its bucket has none (the default 256-point shape)."""
        cfg = (_I32 * 6)()
        ms = ctypes.c_double()
        _raise(self.h, load().ebc_tune_query(_P(self.h), cfg, ctypes.byref(ms)))
        if cfg[0] == 0:
            return None
        return {"bn": cfg[0], "na": cfg[1], "ns": cfg[2], "chunk": cfg[3], "turns": cfg[4], "es": cfg[5],
                "ms": ms.value}

    def save_state(self) -> bytes:
        """Snapshot of the Greedy state (m_v, S, f, counters) as bytes."""
        size = ctypes.c_int64()
        _raise(self.h, load().ebc_state_size(_P(self.h), ctypes.byref(size)))
        buf = (ctypes.c_uint8 * size.value)()
        _raise(self.h, load().ebc_state_save(_P(self.h), ctypes.cast(buf, _P), size.value))
        return bytes(buf)

    def load_state(self, snap: bytes):
        buf = (ctypes.c_uint8 * len(snap)).from_buffer_copy(snap)
        _raise(self.h, load().ebc_state_load(_P(self.h), ctypes.cast(buf, _P), len(snap)))

    def set_precision(self, precision: str, refine_k: int = 8):
        ebc_set_precision(self.h, PRECISIONS[precision], refine_k)
        self.precision = precision

    def greedy(self, k: int):
        """Device outputs: (idx int32[k], f float64[k]) CUDA tensors."""
        import torch
        idx = torch.empty(k, dtype=torch.int32, device="cuda")
        f = torch.empty(k, dtype=torch.float64, device="cuda")
        ebc_greedy(self.h, k, idx.data_ptr(), f.data_ptr())
        return idx, f

    def greedy_host(self, k: int):
        return ebc_greedy_host(self.h, k)

    def gains(self, cand=None):
        import torch
        if cand is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
            ebc_gains(self.h, None, self.n, out.data_ptr())
            return out
        cand = cand.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(cand.numel(), dtype=torch.float64, device="cuda")
        ebc_gains(self.h, cand.data_ptr(), cand.numel(), out.data_ptr())
        self._keep = cand
        return out

    def eval_sets(self, idx, off):
        import torch
        idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
        off = off.to(device="cuda", dtype=torch.int64).contiguous()
        l = off.numel() - 1
        out = torch.empty(max(l, 0), dtype=torch.float64, device="cuda")
        ebc_eval_sets(self.h, idx.data_ptr(), off.data_ptr(), l, out.data_ptr())
        self._keep = (idx, off)
        return out

    def eval_sets_host(self, idx, off):
        return ebc_eval_sets_host(self.h, idx, off)

    def gains_host(self, cand=None):
        return ebc_gains_host(self.h, cand, self.n if cand is None else None)

    def reset(self):
        ebc_reset(self.h)

    def reload(self, V):
        """Replace V (same n, d): torch tensor (host or CUDA) or numpy array."""
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float32)
            assert V.shape == (self.n, self.d)
            ebc_reload(self.h, V.ctypes.data, False)
            self._keep = V
        else:
            assert tuple(V.shape) == (self.n, self.d) and V.is_contiguous()
            ebc_reload(self.h, V.data_ptr(), V.is_cuda)
            self._keep = V

    def profiling(self, on: bool = True):
        ebc_set_profiling(self.h, on)

    def profile(self):
        return ebc_get_profile(self.h)

    def reset_profile(self):
        ebc_reset_profile(self.h)

    def sync(self):
        ebc_sync(self.h)

    def stats(self):
        return ebc_get_stats(self.h)

    def current_f(self):
        return ebc_current_f(self.h)

    def last_round_candidates(self) -> np.ndarray:
        return ebc_last_round_candidates(self.h)

    def reserve_sets(self, max_sets: int, max_members: int):
        """Buffers of ebc_eval_sets for up to max_sets sets / max_members members
        (tensor-core precisions): such calls read nothing back to the host."""
        _raise(self.h, load().ebc_reserve_sets(_P(self.h), int(max_sets), int(max_members)))

    def gain_bounds_host(self, cand=None) -> np.ndarray:
        """Rigorous upper bounds of the gains of ``cand`` (all points if None)
        relative to the current state (ebc_gain_bounds_host)."""
        if cand is None:
            out = np.zeros(self.n, dtype=np.float64)
            _raise(self.h, load().ebc_gain_bounds_host(_P(self.h), None, self.n, out.ctypes.data_as(_P)))
            return out
        cand = np.ascontiguousarray(cand, dtype=np.int32).ravel()
        out = np.zeros(cand.size, dtype=np.float64)
        _raise(self.h, load().ebc_gain_bounds_host(_P(self.h), cand.ctypes.data_as(_P), cand.size,
                                                   out.ctypes.data_as(_P)))
        return out

    def singleton_bounds(self) -> np.ndarray:
        """Upper bounds of every point's gain valid for every S: the bounds
        at S = {} (the current state is saved and restored)."""
        snap = self.save_state()
        try:
            self.reset()
            return self.gain_bounds_host()
        finally:
            self.load_state(snap)

    def max_singleton(self) -> float:
        """max_e f({e}) over V: the exact gain of Greedy's first pick from
        S = {} (the current state is saved and restored)."""
        snap = self.save_state()
        try:
            self.reset()
            return float(self.greedy_host(1)[1][0])
        finally:
            self.load_state(snap)

    def sieve(self, K: int, thresholds, patience: int = 0, bounds=None) -> "Sieve":
        return Sieve(self, K, thresholds, patience, bounds)


class Sieve:
    """Threshold sieve over a stream on one Instance (ebc_sieve_host): feed
    items in pieces; the level / rejection state carries over."""

    def __init__(self, inst: Instance, K: int, thresholds, patience: int = 0, bounds=None):
        self.inst = inst
        self.thr = np.ascontiguousarray(thresholds, dtype=np.float64).ravel()
        self.state = ebc_sieve_state()
        self.state.K = int(K)
        self.state.nthr = self.thr.size
        self.state.thr = self.thr.ctypes.data
        self.state.patience = int(patience)
        self.bounds = None
        if bounds is not None:
            self.bounds = np.ascontiguousarray(bounds, dtype=np.float64).ravel()
            assert self.bounds.size == inst.n
            self.state.bounds = self.bounds.ctypes.data
        self.idx = []
        self.f = []

    def feed(self, items):
        idx, f = ebc_sieve_host(self.inst.h, self.state, items)
        self.idx.extend(idx.tolist())
        self.f.extend(f.tolist())
        return idx, f

    @property
    def level(self) -> int:
        return int(self.state.level)

    @property
    def rejections(self) -> int:
        return int(self.state.rejections)

    def counters(self) -> dict:
        s = self.state
        return {"level": s.level, "rejections": s.rejections, "consumed": s.consumed, "bounded": s.bounded,
                "exact": s.exact}


def three_sieves(inst: Instance, items, K: int, eps: float, T: int, m_single: float | None = None,
                 bounds=None):
    """Three Sieves on the instance's current state: thresholds from K m down
    to m, moving down after T consecutive rejections.  ``bounds``: optional
    upper bounds of every point's gain (e.g. ``inst.singleton_bounds()``).
    Returns (idx, f, Sieve)."""
    if m_single is None:
        m_single = inst.max_singleton()
    sv = Sieve(inst, K, ebc_threshold_ladder(m_single, K, eps, 1.0), T, bounds)
    idx, f = sv.feed(items)
    return idx, f, sv


def sieve_streaming(inst: Instance, items, K: int, eps: float, m_single: float | None = None,
                    workers: int = 1, V=None):
    """Sieve Streaming with the largest singleton value m known: one sieve per
    ladder value up to 2 K m, each run from S = {} over the whole stream; the
    summary of largest f wins (the first such threshold on ties).  Returns
    (best idx, best f, per-sieve f_end list, thresholds); ``inst`` is left in
    the best sieve's state.

    ``workers`` > 1 runs the sieves on that many instances at once (one CUDA
    stream and one host thread each; the binding releases the interpreter
    lock in every library call); ``V`` (the instance's ground set, host array
    or CUDA tensor) is then needed to create them.  Results do not depend on
    ``workers``."""
    if m_single is None:
        m_single = inst.max_singleton()
    thr = ebc_threshold_ladder(m_single, K, eps, 2.0)
    items = np.ascontiguousarray(items, dtype=np.int32).ravel()
    ub0 = inst.singleton_bounds()  # valid for every sieve's S
    ends = [0.0] * thr.size
    snaps = [None] * thr.size
    idxs = [None] * thr.size
    fs = [None] * thr.size

    def run(h_inst, js):
        for j in js:
            h_inst.reset()
            idx, f = Sieve(h_inst, K, [thr[j]], 0, ub0).feed(items)
            ends[j] = float(f[-1]) if f.size else 0.0
            idxs[j], fs[j] = idx, f
            snaps[j] = h_inst.save_state()

    workers = max(1, min(int(workers), thr.size))
    if workers == 1:
        run(inst, range(thr.size))
    else:
        import threading

        import torch
        if V is None:
            raise ValueError("sieve_streaming with workers > 1 needs V")
        streams = [torch.cuda.Stream() for _ in range(workers - 1)]
        pool = [inst] + [Instance(V, precision=inst.precision, stream=st) for st in streams]
        try:
            errs = []

            def body(w):
                try:
                    run(pool[w], range(w, thr.size, workers))
                except Exception as e:  # re-raised below
                    errs.append(e)

            ts = [threading.Thread(target=body, args=(w,)) for w in range(workers)]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
            if errs:
                raise errs[0]
        finally:
            for extra in pool[1:]:
                extra.close()
    best = max(range(thr.size), key=lambda j: (ends[j], -j))
    inst.load_state(snaps[best])
    return idxs[best], fs[best], ends, thr

# ---------------------------------------------------------------------------
# batch runtime (marshalling only)
# ---------------------------------------------------------------------------

def ebc_release_cached_memory() -> None:
    """Return the library pool's cached, unused device memory (current device)."""
    rc = load().ebc_release_cached_memory()
    if rc != EBC_OK:
        raise EbcError(rc, "ebc_release_cached_memory")


def ebc_estimate_bytes(n: int, d: int, prec: int) -> int:
    return int(load().ebc_estimate_bytes(int(n), int(d), int(prec)))


class Group:
    """Greedy on many instances with one persistent bulk launch per round
    (include/ebc.h, ebc_group_*)."""

    def __init__(self, lanes: int = 1, by_row_width: bool = False, max_ctas: int = 0):
        h = _P()
        rc = load().ebc_group_create(ctypes.byref(h))
        if rc != EBC_OK:
            raise EbcError(rc, "ebc_group_create")
        self.h = h.value
        self._err(load().ebc_group_set_lanes(_P(self.h), int(lanes)))
        self._err(load().ebc_group_set_lanes_by_row_width(_P(self.h), int(bool(by_row_width))))
        self._err(load().ebc_group_set_max_ctas(_P(self.h), int(max_ctas)))

    def profiling(self, on: bool = True):
        self._err(load().ebc_group_set_profiling(_P(self.h), int(bool(on))))

    def profile(self) -> dict:
        ms, gap, pairs = ctypes.c_double(), ctypes.c_double(), _I64()
        self._err(load().ebc_group_profile(_P(self.h), ctypes.byref(ms), ctypes.byref(gap), ctypes.byref(pairs)))
        return {"launch_ms": ms.value, "gap_ms": gap.value, "pairs": pairs.value}

    def reset_profile(self):
        self._err(load().ebc_group_reset_profile(_P(self.h)))

    def _err(self, rc):
        if rc != EBC_OK:
            m = load().ebc_group_last_error(_P(self.h))
            raise EbcError(rc, m.decode() if m else "")

    def greedy(self, instances, ks):
        """Enqueue k rounds on every instance; returns per-instance device
        tensors (idx int32[k], f float64[k]), valid once each instance's
        stream reaches them (Instance.sync)."""
        import torch
        n = len(instances)
        outs = [(torch.empty(max(int(k), 1), dtype=torch.int32, device="cuda"),
                 torch.empty(max(int(k), 1), dtype=torch.float64, device="cuda")) for k in ks]
        harr = (_P * n)(*[inst.h for inst in instances])
        karr = (_I32 * n)(*[int(k) for k in ks])
        iarr = (_P * n)(*[o[0].data_ptr() for o in outs])
        farr = (_P * n)(*[o[1].data_ptr() for o in outs])
        self._err(load().ebc_group_greedy(_P(self.h), ctypes.cast(harr, _P), n, ctypes.cast(karr, _P),
                                          ctypes.cast(iarr, _P), ctypes.cast(farr, _P)))
        self._keep = outs
        return [(o[0][:int(k)], o[1][:int(k)]) for o, k in zip(outs, ks)]

    def greedy_host(self, instances, ks):
        """As greedy, then wait for every instance; numpy results."""
        outs = self.greedy(instances, ks)
        res = []
        for inst, (i, f) in zip(instances, outs):
            inst.sync()
            res.append((i.cpu().numpy(), f.cpu().numpy()))
        return res

    def stats(self) -> dict:
        a, b, c = _I64(), _I64(), _I64()
        self._err(load().ebc_group_stats(_P(self.h), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"launches": a.value, "units": b.value, "rounds": c.value}

    def close(self):
        if getattr(self, "h", None):
            load().ebc_group_destroy(_P(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent Greedy summaries sharing the GPU (include/ebc.h, batch runtime)."""

    def __init__(self, max_slots: int = 32, budget_bytes: int = 150 << 30, refine_k: int = 8):
        h = _P()
        rc = load().ebc_batch_create(int(max_slots), int(budget_bytes), int(refine_k), ctypes.byref(h))
        if rc != EBC_OK:
            raise EbcError(rc, "ebc_batch_create")
        self.h = h.value
        self._k = {}

    def _err(self, rc):
        if rc != EBC_OK:
            m = load().ebc_batch_last_error(_P(self.h))
            raise EbcError(rc, m.decode() if m else "")

    def submit(self, V: np.ndarray, k: int, precision: str = "bf16") -> int:
        V = np.ascontiguousarray(V, dtype=np.float32)
        t = _I64()
        self._err(load().ebc_batch_submit(_P(self.h), V.ctypes.data_as(_P), V.shape[0], V.shape[1], int(k),
                                          PRECISIONS[precision], ctypes.byref(t)))
        self._k[t.value] = int(k)
        return t.value

    def set_large(self, large_n: int, max_ctas: int, max_active: int = 0):
        self._err(load().ebc_batch_set_large(_P(self.h), int(large_n), int(max_ctas), int(max_active)))

    def set_autotune(self, reps: int = 3):
        self._err(load().ebc_batch_set_autotune(_P(self.h), int(reps)))

    def set_lazy(self, on: bool = True, min_n: int = 0):
        self._err(load().ebc_batch_set_lazy(_P(self.h), int(bool(on)), int(min_n)))

    def step(self):
        a, q = _I32(), _I32()
        self._err(load().ebc_batch_step(_P(self.h), ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, ticket: int):
        """(idx, f) when finished, else None.  Raises the request's error status."""
        k = self._k[ticket]
        idx = np.zeros(k, np.int32)
        f = np.zeros(k, np.float64)
        done = _I32()
        rc = load().ebc_batch_poll(_P(self.h), int(ticket), idx.ctypes.data_as(_P), f.ctypes.data_as(_P), k,
                                   ctypes.byref(done))
        if done.value:
            del self._k[ticket]
        self._err(rc)
        return (idx, f) if done.value else None

    def run(self):
        self._err(load().ebc_batch_run(_P(self.h)))

    def stats(self) -> dict:
        s = ebc_batch_info()
        self._err(load().ebc_batch_stats(_P(self.h), ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ebc_batch_info._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().ebc_batch_destroy(_P(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
