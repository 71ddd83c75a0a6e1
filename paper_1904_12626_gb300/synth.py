"""Seeded synthetic inputs for the matrix-profile joins.

This module only draws numbers: it holds none of the matrix-profile
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from it.  Every generator takes an explicit integer seed and uses NumPy's
``default_rng`` so the same call gives the same series on every machine.

The recipes follow the workloads the library is measured on (random walks of
the kind the paper's speed experiment uses, Sec. 4 "Speed"; planted motif
pairs and a discord, the properties of Sec. 2; constant stretches that
exercise the zero-variance convention; ragged batches; a pan window set).
"""
from __future__ import annotations

import numpy as np


def random_walk(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """cumsum of N(0,1) steps, length n."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal(n)).astype(dtype)


def pm1_walk(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """cumsum of +-1 steps (the shape of the paper's Sec. 4 speed data)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.choice(np.array([-1.0, 1.0]), size=n)).astype(dtype)


def _spaced_starts(rng, n: int, count: int, length: int, gap: int) -> np.ndarray:
    """`count` start positions of segments of `length` inside [gap, n-length-gap),
    pairwise at least `length + gap` apart (rejection sampling)."""
    starts: list[int] = []
    lo, hi = gap, n - length - gap
    tries = 0
    while len(starts) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place segments")
        s = int(rng.integers(lo, hi))
        if all(abs(s - t) >= length + gap for t in starts):
            starts.append(s)
    return np.array(starts, dtype=np.int64)


def planted_walk(n: int, m: int, seed: int, n_pairs: int = 3, dtype=np.float32):
    """Random walk with `n_pairs` planted motif pairs and one planted discord.

    Motif member: A*sin(2*pi*3*t/m + phi) + level + b + N(0, 0.01^2) noise,
    A ~ U[0.5, 2] and b ~ U[-5, 5] drawn per member, phi shared by the pair,
    `level` the walk's value just before the segment.  Discord: level plus
    3*N(0,1) white noise over m samples.  Segments sit at least 2m apart.

    Returns (x, info) with info = {"pairs": [(p1, p2), ...], "discord": s}.
    """
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal(n))
    starts = _spaced_starts(rng, n, 2 * n_pairs + 1, m, 2 * m)
    t = np.arange(m, dtype=np.float64)
    pairs = []
    for p in range(n_pairs):
        phi = rng.uniform(0.0, 2.0 * np.pi)
        members = (int(starts[2 * p]), int(starts[2 * p + 1]))
        for s in members:
            amp = rng.uniform(0.5, 2.0)
            off = rng.uniform(-5.0, 5.0)
            level = x[s - 1]
            x[s:s + m] = (amp * np.sin(2.0 * np.pi * 3.0 * t / m + phi)
                          + level + off + rng.normal(0.0, 0.01, m))
        pairs.append(members)
    d = int(starts[-1])
    x[d:d + m] = x[d - 1] + 3.0 * rng.standard_normal(m)
    return x.astype(dtype), {"pairs": pairs, "discord": d}


def mixed_with_flats(n: int, m: int, seed: int, block: int = 4096,
                     n_flat: int = 10, flat_len: int | None = None,
                     dtype=np.float32):
    """Series built from `block`-sample blocks, each 50/50 white N(0,1) or a
    random-walk segment continuing from the previous level; then `n_flat`
    non-overlapping constant stretches of `flat_len` (default 2m) samples,
    each equal to the sample just before it.

    Returns (x, flat_starts)."""
    rng = np.random.default_rng(seed)
    flat_len = 2 * m if flat_len is None else flat_len
    out = np.empty(n, dtype=np.float64)
    level = 0.0
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        if rng.random() < 0.5:
            seg = rng.standard_normal(b1 - b0)
        else:
            seg = level + np.cumsum(rng.standard_normal(b1 - b0))
            level = seg[-1]
        out[b0:b1] = seg
    starts = np.sort(_spaced_starts(rng, n, n_flat, flat_len, m))
    for s in starts:
        out[s:s + flat_len] = out[s - 1]
    return out.astype(dtype), starts


def ragged_batch(n_series: int, seed: int, len_lo: int = 1000, len_hi: int = 65536,
                 windows=(32, 64, 128), dtype=np.float32):
    """`n_series` random walks with lengths ~ U{len_lo..len_hi} and a window
    per series drawn from `windows`, concatenated.

    Returns (values, offsets[n_series+1] int64, ms[n_series] int32)."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(len_lo, len_hi + 1, size=n_series).astype(np.int64)
    ms = rng.choice(np.asarray(windows, dtype=np.int32), size=n_series).astype(np.int32)
    offsets = np.zeros(n_series + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    steps = rng.standard_normal(int(offsets[-1]))
    values = np.empty(int(offsets[-1]), dtype=np.float64)
    for s in range(n_series):
        a, b = offsets[s], offsets[s + 1]
        values[a:b] = np.cumsum(steps[a:b])
    return values.astype(dtype), offsets, ms


def pan_windows(count: int = 64, lo: int = 16, hi: int = 1024) -> np.ndarray:
    """`count` window sizes spaced geometrically from lo to hi, rounded to the
    nearest integer (Python round-half-even)."""
    ratio = hi / lo
    ws = [int(round(lo * ratio ** (k / (count - 1)))) for k in range(count)]
    return np.asarray(ws, dtype=np.int32)


def sample_rows(l: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct row indices in [0, l), sorted (all rows if count >= l)."""
    if count >= l:
        return np.arange(l, dtype=np.int64)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(l, size=count, replace=False)).astype(np.int64)


def tonal(n: int, seed: int = 0, dtype=np.float64, n_tones: int = 4) -> np.ndarray:
    """A bounded, music-like signal for the non-normalised distance (SiMPle's
    domain, Sec. 3.3.4): a few sinusoids whose amplitudes drift slowly, plus
    N(0, 0.05^2) noise; values stay within a few units of zero."""
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64)
    x = np.zeros(n)
    for _ in range(n_tones):
        period = rng.uniform(12.0, 200.0)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        amp = 0.5 + 0.5 * np.sin(2.0 * np.pi * t / rng.uniform(5000.0, 50000.0) + rng.uniform(0, 6.3))
        x += amp * np.sin(2.0 * np.pi * t / period + phase)
    x += 0.05 * rng.standard_normal(n)
    return x.astype(dtype)
