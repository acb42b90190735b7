"""Seeded synthetic inputs for the DTW retrieval cascade.

This module only draws numbers: it holds none of the method's arithmetic
(no envelope, bound or DTW).  The CUDA path and the FP64 oracle both take
their inputs from here, so the two sides see the same fp32 arrays.

Every generator is deterministic in (seed, stream): a `numpy.random.PCG64`
generator is derived from `SeedSequence([seed, stream, chunk])`, and large
draws are made in fixed chunks of rows so that the output does not depend
on how much memory the caller has.

Workloads (Sec. 10 of the paper describes the originals):

* random walks, x_1 = 0 and x_i = x_{i-1} + N(0,1)  (Sec. 10.1);
* shape-like series: a class pattern (flat plateau, rising ramp, falling
  ramp, or a sum of 1-3 sinusoids with random phase) plus N(0, 0.1) noise,
  shifted in time by up to 10 % of n with edge-value padding, then
  z-normalised.  These stand in for the shape archive and the
  Cylinder-Bell-Funnel style sets of Sec. 10, which are not available; the
  patterns are designed here from that description, not taken from any
  published generator.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "random_walks",
    "shapes",
    "shape_classes",
    "SHAPE_CLASSES",
    "bucket_lengths",
    "log_uniform_lengths",
    "STREAM_DB",
    "STREAM_QUERY",
]

# Distinct seed streams: database rows and queries never share draws.
STREAM_DB = 0
STREAM_QUERY = 1

_CHUNK = 1 << 15  # rows per independent draw


def _rng(seed: int, stream: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, chunk])))


def random_walks(count: int, n: int, seed: int, stream: int = STREAM_DB) -> np.ndarray:
    """`count` random walks of length `n` as a C-contiguous fp32 [count, n] array.

    x_1 = 0 and x_i = x_{i-1} + N(0, 1), accumulated in fp64 and rounded
    once to fp32 (Sec. 10.1).
    """
    if count < 0 or n < 1:
        raise ValueError("count >= 0 and n >= 1 required")
    out = np.empty((count, n), dtype=np.float32)
    for c, lo in enumerate(range(0, count, _CHUNK)):
        hi = min(count, lo + _CHUNK)
        steps = _rng(seed, stream, c).standard_normal((hi - lo, n))
        steps[:, 0] = 0.0
        out[lo:hi] = np.cumsum(steps, axis=1)
    return out


SHAPE_CLASSES = 4  # plateau, rising ramp, falling ramp, sum of sinusoids


def _shape_rows(g: np.random.Generator, rows: int, n: int, cls=None) -> np.ndarray:
    t = np.arange(n, dtype=np.float64)
    out = np.empty((rows, n), dtype=np.float64)
    if cls is None:
        cls = g.integers(0, SHAPE_CLASSES, size=rows)
    for r in range(rows):
        c = int(cls[r])
        if c < 3:
            # an event [a, b) of random position and length and a height
            a = int(g.integers(n // 8, n // 4 + 1))
            b = int(g.integers(a + max(1, n // 4), a + max(2, (3 * n) // 4) + 1))
            b = min(b, n)
            h = 6.0 + g.standard_normal()
            s = np.zeros(n)
            span = max(1, b - a)
            if c == 0:  # flat plateau
                s[a:b] = h
            elif c == 1:  # rising ramp
                s[a:b] = h * (t[a:b] - a) / span
            else:  # falling ramp
                s[a:b] = h * (b - t[a:b]) / span
        else:  # sum of 1-3 sinusoids with random phase
            s = np.zeros(n)
            for _ in range(int(g.integers(1, 4))):
                cycles = g.uniform(0.5, 8.0)
                amp = g.uniform(0.5, 2.0)
                phase = g.uniform(0.0, 2.0 * np.pi)
                s += amp * np.sin(2.0 * np.pi * cycles * t / n + phase)
        s = s + 0.1 * g.standard_normal(n)
        # integer time shift with edge-value padding (not circular)
        m = n // 10
        sh = int(g.integers(-m, m + 1)) if m > 0 else 0
        if sh > 0:
            s = np.concatenate([np.full(sh, s[0]), s[: n - sh]])
        elif sh < 0:
            s = np.concatenate([s[-sh:], np.full(-sh, s[-1])])
        mu = s.mean()
        sd = s.std()
        out[r] = (s - mu) / sd if sd > 0 else s - mu
    return out


def white_noise(count: int, n: int, seed: int, stream: int = STREAM_DB) -> np.ndarray:
    """`count` white-noise series x_i = N(0, 1) of length `n` (App. B), fp32 [count, n]."""
    if count < 0 or n < 1:
        raise ValueError("count >= 0 and n >= 1 required")
    out = np.empty((count, n), dtype=np.float32)
    step = max(1, (1 << 22) // n)
    for k, r0 in enumerate(range(0, count, step)):
        r1 = min(count, r0 + step)
        out[r0:r1] = _rng(seed, stream, (1 << 21) + k).standard_normal((r1 - r0, n))
    return out


def shapes(count: int, n: int, seed: int, stream: int = STREAM_DB) -> np.ndarray:
    """`count` shape-like series of length `n`, fp32 [count, n], z-normalised in fp64."""
    if count < 0 or n < 1:
        raise ValueError("count >= 0 and n >= 1 required")
    out = np.empty((count, n), dtype=np.float32)
    for c, lo in enumerate(range(0, count, _CHUNK)):
        hi = min(count, lo + _CHUNK)
        out[lo:hi] = _shape_rows(_rng(seed, stream, c), hi - lo, n)
    return out


def shape_classes(labels, n: int, seed: int, stream: int = STREAM_DB) -> np.ndarray:
    """Shape-like series of the given classes (0 plateau, 1 rising ramp, 2
    falling ramp, 3 sum of sinusoids), fp32 [len(labels), n]: the labelled
    stand-in for the classification experiment of App. C."""
    labels = np.asarray(labels, dtype=np.int64)
    if labels.ndim != 1 or np.any((labels < 0) | (labels >= SHAPE_CLASSES)) or n < 1:
        raise ValueError("labels in [0, %d) and n >= 1 required" % SHAPE_CLASSES)
    out = np.empty((labels.shape[0], n), dtype=np.float32)
    for c, lo in enumerate(range(0, labels.shape[0], _CHUNK)):
        hi = min(labels.shape[0], lo + _CHUNK)
        out[lo:hi] = _shape_rows(_rng(seed, stream + 32, c), hi - lo, n, cls=labels[lo:hi])
    return out


def bucket_lengths(lo: int = 64, hi: int = 2048) -> list[int]:
    """Length buckets at lo * 2^(j/2), rounded, from lo up to hi inclusive."""
    out = []
    j = 0
    while True:
        v = int(round(lo * 2.0 ** (j / 2.0)))
        if v > hi:
            break
        out.append(v)
        j += 1
    return out


def log_uniform_lengths(count: int, lo: int, hi: int, seed: int, stream: int = STREAM_QUERY) -> np.ndarray:
    """Query lengths drawn log-uniformly in [lo, hi] (int64)."""
    g = _rng(seed, stream, 1 << 20)
    v = np.exp(g.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def snap_to_buckets(lengths, buckets) -> np.ndarray:
    """Each length replaced by the bucket nearest to it in log space (int64)."""
    lb = np.log(np.asarray(buckets, dtype=np.float64))
    ll = np.log(np.asarray(lengths, dtype=np.float64))
    j = np.argmin(np.abs(ll[:, None] - lb[None, :]), axis=1)
    return np.asarray(buckets, dtype=np.int64)[j]


def mixed_queries(lengths, seed: int, stream: int = STREAM_QUERY) -> list[np.ndarray]:
    """One random walk per requested length (fp32 1-D arrays), drawn per length
    bucket in order of appearance so that the values do not depend on the batch."""
    lengths = np.asarray(lengths, dtype=np.int64)
    out: list[np.ndarray] = [None] * len(lengths)  # type: ignore[list-item]
    for n in np.unique(lengths):
        pos = np.flatnonzero(lengths == n)
        rows = random_walks(len(pos), int(n), seed=seed * 7919 + int(n), stream=stream)
        for r, i in enumerate(pos):
            out[i] = rows[r]
    return out


def poisson_arrivals(count: int, rate: float, seed: int, stream: int = STREAM_QUERY) -> np.ndarray:
    """Arrival times (seconds, float64, increasing) of a Poisson process of the given rate."""
    g = _rng(seed, stream, (1 << 20) + 1)
    return np.cumsum(g.exponential(1.0 / rate, size=count))
