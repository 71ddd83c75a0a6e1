"""The synthetic input recipes (no GPU): every generator is deterministic
for its seed and produces the structure the workloads are described with --
planted motif pairs and a discord at least 2m apart, flat stretches of 2m
samples, ragged lengths and windows in range, and the 64 geometric pan
window sizes.  The motif and discord checks go through the oracle, so they
also show the planted structure is what a matrix profile sees."""
import math

import numpy as np

import oracle
from paper_1904_12626_gb300 import synth


def test_seeded_and_shaped():
    for gen in (lambda s: synth.random_walk(5000, seed=s), lambda s: synth.pm1_walk(5000, seed=s),
                lambda s: synth.tonal(5000, seed=s)):
        a, b, c = gen(1), gen(1), gen(2)
        assert a.shape == (5000,) and np.array_equal(a, b) and not np.array_equal(a, c)
    w = synth.random_walk(200000, seed=3)
    assert abs(np.std(np.diff(w)) - 1.0) < 0.01                 # N(0, 1) steps
    p = synth.pm1_walk(10000, seed=3)
    assert set(np.unique(np.diff(p))) <= {-1.0, 1.0}
    assert synth.random_walk(10, seed=0, dtype=np.float32).dtype == np.float32
    t = synth.tonal(100000, seed=4)
    assert np.isfinite(t).all() and np.abs(t).max() < 5.0


def test_planted_walk_structure():
    n, m = 40000, 64
    x, info = synth.planted_walk(n, m, seed=5)
    x2, info2 = synth.planted_walk(n, m, seed=5)
    assert np.array_equal(x, x2) and info == info2 and x.dtype == np.float32
    starts = sorted([p for pair in info["pairs"] for p in pair] + [info["discord"]])
    assert len(info["pairs"]) == 3 and len(starts) == 7
    assert all(b - a >= 3 * m for a, b in zip(starts, starts[1:]))   # m long, 2m gap
    assert starts[0] >= 2 * m and starts[-1] + m + 2 * m <= n
    x64 = x.astype(np.float64)
    for p1, p2 in info["pairs"]:
        # same shape up to amplitude and offset, noise 0.01: nearly zero distance
        assert oracle.distance(x64, m, p1, p2) < 0.05 * math.sqrt(2 * m)
    # the planted pairs are each other's nearest neighbours, the discord has the largest MP
    rows = np.array(sorted([p for pair in info["pairs"] for p in pair]))
    mp, pi, _ = oracle.selfjoin(x64, m, rows=rows)
    partner = {a: b for pair in info["pairs"] for a, b in (pair, pair[::-1])}
    for r, j in zip(rows, pi):
        assert abs(int(j) - partner[int(r)]) <= 2
    # the discord's nearest neighbour is farther than that of any of 50 sampled windows
    d = info["discord"]
    sample = [int(r) for r in synth.sample_rows(n - m + 1, 60, seed=9) if abs(int(r) - d) >= m][:50]
    mp_d, _, _ = oracle.selfjoin(x64, m, rows=np.array([d]))
    mp_s, _, _ = oracle.selfjoin(x64, m, rows=np.array(sample))
    assert mp_d[0] > mp_s.max()


def test_mixed_with_flats_structure():
    n, m = 60000, 32
    x, flats = synth.mixed_with_flats(n, m, seed=6)
    assert x.shape == (n,) and len(flats) == 10 and np.all(np.diff(flats) >= 2 * m + m)
    for s in flats:
        seg = x[s - 1:s + 2 * m]
        assert np.all(seg == seg[0])                          # 2m samples equal to the one before
    # blocks of 4096: some white (no drift), some walks
    steps = [np.std(np.diff(x[b:b + 4096].astype(np.float64))) for b in range(0, n - 4096, 4096)]
    assert min(steps) < 1.2 and max(steps) > 1.2


def test_ragged_batch_ranges():
    values, offsets, ms = synth.ragged_batch(300, seed=7)
    lens = np.diff(offsets)
    assert offsets[0] == 0 and offsets[-1] == len(values) and len(ms) == 300
    assert lens.min() >= 1000 and lens.max() <= 65536
    assert set(np.unique(ms)) <= {32, 64, 128} and len(np.unique(ms)) == 3
    assert ms.dtype == np.int32 and offsets.dtype == np.int64
    # each series starts a fresh walk: its first value is one N(0, 1) step
    assert np.abs(values[offsets[:-1]]).max() < 5.0


def test_pan_windows_reading():
    """64 sizes round(16 * 64^(k/63)), Python rounding: distinct, 16..1024."""
    ws = synth.pan_windows()
    assert len(ws) == 64 and len(set(ws.tolist())) == 64
    assert ws[0] == 16 and ws[-1] == 1024 and np.all(np.diff(ws) > 0)
    assert ws.tolist()[:4] == [16, 17, 18, 20]
    ratios = ws[1:] / ws[:-1]
    assert np.all(np.abs(ratios - 64 ** (1 / 63)) < 0.06)


def test_sample_rows():
    r = synth.sample_rows(1000, 50, seed=8)
    assert len(r) == 50 and len(np.unique(r)) == 50 and np.all(np.diff(r) > 0)
    assert r.min() >= 0 and r.max() < 1000
    assert np.array_equal(synth.sample_rows(10, 20, seed=8), np.arange(10))
