"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and lays out locations; it holds none of the
likelihood arithmetic (no covariance, factorisation or solve), so both the CPU
oracle and the CUDA path can take their inputs from it without sharing any of
the method's code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: value k of
stream (seed, tag) is mix64(base(seed, tag) + (k + 1) * GOLDEN).  Normal
variates use the Box-Muller transform (Box & Muller, 1958).

Locations follow the paper's synthetic workload (Section 7.1): an m x m grid
over the unit square, point (r, l) at ((r - 0.5 + X_rl) / m, (l - 0.5 + Y_rl) / m)
with X, Y ~ U(-0.4, 0.4), r, l = 1..m.  The paper prints the scale as n^{1/2};
it is read as n^{-1/2} = 1/m so that the points lie in [0, 1]^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAG_MULT = np.uint64(0xD1B54A32D192ED03)

# Stream tags: each tag is an independent counter stream for a given seed.
TAG_JITTER_X = 0
TAG_JITTER_Y = 1
TAG_NORMAL = 2
TAG_BATCH = 3
TAG_SUBSQUARE = 4


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = z.astype(np.uint64, copy=True)
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _stream_base(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        return np.uint64(s ^ (np.uint64(tag) * _TAG_MULT))


def raw_u64(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-mode SplitMix64: values offset..offset+count-1 of stream (seed, tag)."""
    base = _stream_base(seed, tag)
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(base + k * GOLDEN)


def uniform(seed: int, tag: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (raw_u64(seed, tag, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, tag: int = TAG_NORMAL) -> np.ndarray:
    """Standard normal variates by Box-Muller from pairs of uniforms."""
    pairs = (count + 1) // 2
    u = uniform(seed, tag, 2 * pairs)
    u1 = 1.0 - u[0::2]  # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * pairs)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


def jittered_grid(n: int, seed: int = 0, origin=(0.0, 0.0), side: float = 1.0) -> np.ndarray:
    """n locations on a jittered m x m grid, m = ceil(sqrt(n)), row-major order.

    Returns a (2, n) float64 array: row 0 holds x, row 1 holds y.  With the
    default origin and side the grid covers [0, 1]^2; the batched workload
    places it on a sub-square instead.  When n < m*m the first n points are kept.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    m = int(math.isqrt(n))
    if m * m < n:
        m += 1
    jx = uniform(seed, TAG_JITTER_X, n) * 0.8 - 0.4
    jy = uniform(seed, TAG_JITTER_Y, n) * 0.8 - 0.4
    idx = np.arange(n)
    r = (idx // m) + 1
    l = (idx % m) + 1
    locs = np.empty((2, n))
    locs[0] = origin[0] + side * (r - 0.5 + jx) / m
    locs[1] = origin[1] + side * (l - 0.5 + jy) / m
    return locs


@dataclass(frozen=True)
class Problem:
    """One synthetic likelihood problem: locations, theta and the seed of e."""
    n: int
    theta: tuple
    seed: int
    origin: tuple = (0.0, 0.0)
    side: float = 1.0

    def locations(self) -> np.ndarray:
        return jittered_grid(self.n, self.seed, self.origin, self.side)

    def e(self) -> np.ndarray:
        return normal(self.seed, self.n)


# The five workloads.  Sizes and theta follow the paper's synthetic study
# (Section 7.1-7.2: theta = (1, 0.1, 0.5)) and the mixed, batched and serving
# variants built on top of it.
CONFIG1 = Problem(n=1600, theta=(1.0, 0.1, 0.5), seed=0)
CONFIG2 = Problem(n=25600, theta=(1.0, 0.2, 1.3), seed=0)
CONFIG3 = Problem(n=102400, theta=(1.0, 0.1, 0.5), seed=0)


def batched_problems(count: int = 512, seed: int = 0, n_lo: int = 256, n_hi: int = 4096) -> list:
    """Uneven batch: n ~ U{n_lo..n_hi}, theta1 ~ U(0.5, 2), theta2 ~ U(0.03, 0.3),
    theta3 ~ U(0.3, 2); each problem k is a jittered grid on a random
    sub-square (side ~ U(0.2, 1), origin uniform inside [0, 1]^2) with seed k."""
    u = uniform(seed, TAG_BATCH, 6 * count).reshape(count, 6)
    out = []
    for k in range(count):
        n = n_lo + int(u[k, 0] * (n_hi - n_lo + 1))
        n = min(n, n_hi)
        th = (0.5 + 1.5 * u[k, 1], 0.03 + 0.27 * u[k, 2], 0.3 + 1.7 * u[k, 3])
        side = 0.2 + 0.8 * u[k, 4]
        o = uniform(k, TAG_SUBSQUARE, 2) * (1.0 - side)
        out.append(Problem(n=n, theta=th, seed=k, origin=(float(o[0]), float(o[1])), side=side))
        _ = u[k, 5]
    return out


def serving_fields(count: int = 64, seed: int = 1, n_lo: int = 1000, n_hi: int = 40000) -> list:
    """Serving workload: fields with n log-uniform in [n_lo, n_hi], theta3 ~ U(0.3, 2)."""
    u = uniform(seed, TAG_BATCH, 4 * count).reshape(count, 4)
    out = []
    for k in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[k, 0] * (math.log(n_hi) - math.log(n_lo)))))
        th = (0.5 + 1.5 * u[k, 1], 0.03 + 0.27 * u[k, 2], 0.3 + 1.7 * u[k, 3])
        out.append(Problem(n=n, theta=th, seed=1000 + k))
    return out
