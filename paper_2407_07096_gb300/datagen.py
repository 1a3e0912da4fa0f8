"""Seeded synthetic inputs: isotropic Gaussian mixtures for the exact-KDE workloads.

This module holds no KDE arithmetic. It is the one piece shared by the CUDA path's
tests/benchmark and the CPU oracle's tests: both are handed the same arrays.

Generator: SplitMix64 used counter-style (value i of stream s under seed k is
``mix64(key(k, s) + (i + 1) * GOLDEN)``, Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), uniforms from the top 53 bits, normals
by the Box-Muller transform (Box & Muller 1958). Everything is vectorised numpy with
explicit uint64 wrap-around, so the bytes produced do not depend on numpy's own
random-number streams or its version.

Workloads (the paper evaluates on real datasets that are not available here; these
mixtures stand in for them, Sec. 6.1):
  * ``mixture(...)``: K components, means uniform in [lo, hi]^d, per-component std
    either fixed or log-uniform in [s0, s1], component index uniform per point,
    equal weights. Queries come from the same mixture on separate streams.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1

# stream identifiers (arbitrary distinct constants)
S_MEANS, S_STDS, S_COMP_X, S_NOISE_X, S_COMP_Q, S_NOISE_Q, S_AUX = range(1, 8)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK
    z ^= z >> 31
    return z


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of stream ``stream`` under ``seed`` (two chained SplitMix64 mixes)."""
    return _mix64_int(_mix64_int(seed & _MASK) ^ ((stream * 0xD1B54A32D192ED03) & _MASK))


def raw_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Values ``start .. start+count-1`` of the counter-based SplitMix64 stream."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + idx * _GOLDEN)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (raw_u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_open0(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in (0, 1]."""
    return ((raw_u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller; value i uses uniforms 2i and 2i+1 of the stream."""
    p0 = start // 2
    p1 = (start + count + 1) // 2
    u = uniform_open0(seed, stream, 2 * (p1 - p0), 2 * p0)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * math.pi * u[1::2]
    out = np.empty(2 * (p1 - p0), dtype=np.float64)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    off = start - 2 * p0
    return out[off:off + count]


@dataclass(frozen=True)
class Mixture:
    """A K-component isotropic Gaussian mixture in d dimensions."""
    means: np.ndarray  # K x d float64
    stds: np.ndarray   # K float64

    @property
    def d(self) -> int:
        return int(self.means.shape[1])

    @property
    def k(self) -> int:
        return int(self.means.shape[0])


def make_mixture(seed: int, k: int, d: int, lo: float, hi: float,
                 std: float | tuple[float, float] = 1.0) -> Mixture:
    """Means uniform in [lo, hi]^d; std fixed, or log-uniform in [std[0], std[1]]."""
    means = lo + (hi - lo) * uniform(seed, S_MEANS, k * d).reshape(k, d)
    if isinstance(std, tuple):
        s0, s1 = std
        u = uniform(seed, S_STDS, k)
        stds = np.exp(math.log(s0) + u * (math.log(s1) - math.log(s0)))
    else:
        stds = np.full(k, float(std))
    return Mixture(means, stds)


def sample(mix: Mixture, seed: int, count: int, which: str = "data",
           dtype=np.float32, chunk: int = 1 << 20) -> np.ndarray:
    """``count`` points from ``mix``; ``which`` selects the data or the query streams.

    Generated in chunks of rows so that memory stays bounded at large ``count``.
    """
    s_comp, s_noise = (S_COMP_X, S_NOISE_X) if which == "data" else (S_COMP_Q, S_NOISE_Q)
    d = mix.d
    out = np.empty((count, d), dtype=dtype)
    for r0 in range(0, count, chunk):
        r1 = min(count, r0 + chunk)
        comp = np.minimum((uniform(seed, s_comp, r1 - r0, r0) * mix.k).astype(np.int64), mix.k - 1)
        z = normal(seed, s_noise, (r1 - r0) * d, r0 * d).reshape(r1 - r0, d)
        out[r0:r1] = (mix.means[comp] + mix.stds[comp, None] * z).astype(dtype)
    return out


def log_uniform_int(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers log-uniform in [lo, hi]."""
    u = uniform(seed, stream, count)
    v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


# --------------------------------------------------------------------------------------
# The workloads, by their sizes (unspecified details and seeds are stated readings).
# --------------------------------------------------------------------------------------

def workload_small_f64(seed: int = 0):
    """n = m = 1000, d = 2, FP64; 3 components, means in [-5, 5]^2, std 1; a = 1."""
    mix = make_mixture(seed, 3, 2, -5.0, 5.0, 1.0)
    X = sample(mix, seed, 1000, "data", np.float64)
    Q = sample(mix, seed, 1000, "query", np.float64)
    return X, Q, 1.0


def workload_single_d16(seed: int = 0, n: int = 100_000, m: int = 100_000):
    """n = m = 100000, d = 16, FP32; 10 components, means in [-10, 10]^16, std 1."""
    mix = make_mixture(seed, 10, 16, -10.0, 10.0, 1.0)
    return sample(mix, seed, n, "data"), sample(mix, seed, m, "query")


def workload_large_d64(seed: int = 0, n: int = 2_000_000, m: int = 100_000):
    """n = 2e6, m = 1e5, d = 64, FP32; 50 components, means in [-10, 10]^64, std
    log-uniform in [0.5, 2]; a = 0.05."""
    mix = make_mixture(seed, 50, 64, -10.0, 10.0, (0.5, 2.0))
    return sample(mix, seed, n, "data"), sample(mix, seed, m, "query"), 0.05
