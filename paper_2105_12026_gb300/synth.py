"""Seeded synthetic inputs for the exemplar-based clustering workloads.

This module holds input generation only: Gaussian mixtures, drifting
"process regime" features, candidate-set lists and request traces.  It
contains none of the summariser's arithmetic (no distances, no f, no gains),
so both the CUDA path and the CPU oracle may consume what it produces.

Every generator draws in FP64 from numpy's PCG64 (``default_rng``), applies a
per-dimension z-score (population standard deviation, ddof=0; a dimension with
zero spread is left at zero) in FP64 and only then casts to FP32, so the FP32
arrays handed to either side are bit-identical for a given seed.

The paper evaluates on randomly generated problems without stating their
distribution (Sec. 5) and on proprietary injection-moulding cycles (Sec. 6);
the shapes here stand in for both.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np


def zscore_to_f32(x: np.ndarray) -> np.ndarray:
    """Per-dimension z-score in FP64 (ddof=0), then cast to FP32."""
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(axis=0)
    sd = x.std(axis=0)
    out = np.zeros_like(x)
    ok = sd > 0
    out[:, ok] = (x[:, ok] - mu[ok]) / sd[ok]
    return np.ascontiguousarray(out.astype(np.float32))


def gaussian_mixture(rng: np.random.Generator, n: int, d: int, clusters: int,
                     sigma=0.5, anisotropic: bool = False,
                     sigma_range=(0.2, 1.5)) -> np.ndarray:
    """Equal-weight Gaussian mixture, means U[-3,3]^d.

    ``anisotropic`` draws a per-cluster diagonal sigma in ``sigma_range``;
    otherwise ``sigma`` is a scalar (isotropic) or ``None`` to draw one
    isotropic sigma per cluster from ``sigma_range``.
    """
    means = rng.uniform(-3.0, 3.0, size=(clusters, d))
    if anisotropic:
        sig = rng.uniform(sigma_range[0], sigma_range[1], size=(clusters, d))
    elif sigma is None:
        sig = np.repeat(rng.uniform(sigma_range[0], sigma_range[1], size=(clusters, 1)), d, axis=1)
    else:
        sig = np.full((clusters, d), float(sigma))
    lab = rng.integers(0, clusters, size=n)
    x = means[lab] + rng.standard_normal((n, d)) * sig[lab]
    return x


def drift_regimes(rng: np.random.Generator, n: int, d: int, regimes: int = 6,
                  sigma: float = 0.5, outlier_frac: float = 0.02,
                  outlier_sigmas: float = 5.0) -> np.ndarray:
    """Injection-moulding-like cycle features.

    ``regimes`` contiguous, time-ordered runs of about n/regimes points.  Run r
    has mean U[-3,3]^d plus a linear drift (t/T_r)*delta_r, where delta_r is
    sigma*sqrt(d) along a random unit direction (one sigma per dimension in
    RMS), and isotropic noise sigma.  A fraction ``outlier_frac`` of points,
    chosen at random, is moved by outlier_sigmas*sigma*sqrt(d) along a random
    unit direction.
    """
    bounds = np.linspace(0, n, regimes + 1).astype(np.int64)
    x = np.empty((n, d), dtype=np.float64)
    for r in range(regimes):
        a, b = int(bounds[r]), int(bounds[r + 1])
        mu = rng.uniform(-3.0, 3.0, size=d)
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        delta = sigma * np.sqrt(d) * u
        t = (np.arange(b - a, dtype=np.float64) / max(b - a - 1, 1))[:, None]
        x[a:b] = mu + t * delta + sigma * rng.standard_normal((b - a, d))
    n_out = int(round(outlier_frac * n))
    if n_out:
        idx = rng.choice(n, size=n_out, replace=False)
        dirs = rng.standard_normal((n_out, d))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        x[idx] += outlier_sigmas * sigma * np.sqrt(d) * dirs
    return x


def random_sets(rng: np.random.Generator, n: int, l: int, smin: int, smax: int):
    """CSR candidate sets: sizes U{smin..smax}, members without replacement."""
    sizes = rng.integers(smin, smax + 1, size=l)
    off = np.zeros(l + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = np.empty(int(off[-1]), dtype=np.int32)
    for j in range(l):
        idx[off[j]:off[j + 1]] = rng.choice(n, size=int(sizes[j]), replace=False)
    return idx, off


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------
# The five workloads.  Each returns plain numpy arrays.
# --------------------------------------------------------------------------

def plain_greedy_small(seed: int = 0, n: int = 1000, d: int = 16):
    """Greedy, n=1,000, d=16: 8-cluster isotropic GMM (sigma 0.5), k=10."""
    rng = np.random.default_rng(seed)
    V = zscore_to_f32(gaussian_mixture(rng, n, d, 8, sigma=0.5))
    return {"V": V, "k": 10}


def multiset_eval(seed: int = 0, n: int = 50_000, d: int = 64, l: int = 1024,
                  smin: int = 1, smax: int = 64):
    """Multi-set evaluation: 32-cluster anisotropic GMM, l CSR sets of size U{1..64}."""
    ss = np.random.SeedSequence(seed).spawn(2)
    V = zscore_to_f32(gaussian_mixture(np.random.default_rng(ss[0]), n, d, 32,
                                       anisotropic=True))
    idx, off = random_sets(np.random.default_rng(ss[1]), n, l, smin, smax)
    return {"V": V, "idx": idx, "off": off}


def regime_greedy(seed: int = 0, n: int = 200_000, d: int = 128, k: int = 100):
    """Greedy k=100 on drifting-regime features, n=200,000, d=128."""
    rng = np.random.default_rng(seed)
    V = zscore_to_f32(drift_regimes(rng, n, d))
    return {"V": V, "k": k}


def case_study_series(seed: int = 0, n: int = 1_000, d: int = 3_524, regimes: int = 8):
    """Stand-in for the case study's sensor curves (Sec. 6: n = 1,000 cycles
    of d = 3,524 samples each): every regime a template curve
    sum_j a_j sin(2 pi f_j t + p_j) + b t on t in [0, 1] (4 terms, a ~ U[0.5, 2],
    f ~ U{1..20}, p ~ U[0, 2 pi], b ~ U[-1, 1]); cycles come in contiguous
    runs of one regime (random run lengths), each its regime's curve scaled
    by 1 + 0.05 N(0, 1) plus white noise of sigma 0.3; z-scored."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, d)
    tmpl = np.zeros((regimes, d))
    for r in range(regimes):
        a = rng.uniform(0.5, 2.0, 4)
        f = rng.integers(1, 21, 4)
        ph = rng.uniform(0.0, 2 * np.pi, 4)
        tmpl[r] = (a[:, None] * np.sin(2 * np.pi * f[:, None] * t[None, :] + ph[:, None])).sum(0)
        tmpl[r] += rng.uniform(-1.0, 1.0) * t
    cuts = np.sort(rng.choice(np.arange(1, n), size=regimes - 1, replace=False))
    lab = np.zeros(n, dtype=np.int64)
    for r, c in enumerate(cuts):
        lab[c:] = r + 1
    scale = 1.0 + 0.05 * rng.standard_normal(n)
    x = tmpl[lab] * scale[:, None] + 0.3 * rng.standard_normal((n, d))
    return zscore_to_f32(x)


@dataclass
class InstanceSpec:
    n: int
    d: int
    k: int
    clusters: int
    seed: int
    kind: str = "gmm"

    def make(self) -> np.ndarray:
        rng = np.random.default_rng(self.seed)
        if self.kind == "drift":
            return zscore_to_f32(drift_regimes(rng, self.n, self.d))
        return zscore_to_f32(gaussian_mixture(rng, self.n, self.d, self.clusters, sigma=None))


def instance_mix(seed: int = 0, count: int = 256, n_lo: int = 2_000, n_hi: int = 100_000,
                 dims=(16, 32, 64, 128), k_lo: int = 5, k_hi: int = 50):
    """Batched greedy mix: n log-uniform, d from ``dims``, k U{k_lo..k_hi}, 4-64 clusters."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count)).astype(np.int64)
    d = rng.choice(np.asarray(dims), size=count)
    k = rng.integers(k_lo, k_hi + 1, size=count)
    cl = rng.integers(4, 65, size=count)
    child = rng.integers(0, 2**31 - 1, size=count)
    return [InstanceSpec(int(n[i]), int(d[i]), int(k[i]), int(cl[i]), int(child[i]))
            for i in range(count)]


@dataclass
class Request:
    t_arrive: float
    spec: InstanceSpec
    large: bool = False


def request_trace(seed: int = 0, rate: float = 50.0, horizon_s: float = 60.0,
                  large_frac: float = 0.05, large_n: int = 1_000_000, large_d: int = 32,
                  large_k=(10, 200), mix_kwargs=None):
    """Poisson arrivals; a fraction ``large_frac`` are large drift-regime requests."""
    rng = np.random.default_rng(seed)
    mix_kwargs = dict(mix_kwargs or {})
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > horizon_s:
            break
        if rng.random() < large_frac:
            k = int(rng.integers(large_k[0], large_k[1] + 1))
            spec = InstanceSpec(large_n, large_d, k, 6, int(rng.integers(0, 2**31 - 1)), kind="drift")
            reqs.append(Request(t, spec, True))
        else:
            spec = instance_mix(int(rng.integers(0, 2**31 - 1)), count=1, **mix_kwargs)[0]
            reqs.append(Request(t, spec, False))
    return reqs
