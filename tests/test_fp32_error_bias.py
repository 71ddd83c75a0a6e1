"""The FP32-mixed path's error bias, checked against emulated FP32 rounding
(no GPU).

The tile kernel walks each diagonal with the covariance recurrence
c(i,j) = c(i-1,j-1) + df_i dg_j + df_j dg_i in FP32 (two fused multiply-adds
per cell, operands rounded to FP32) from an exact anchor, and adds to every
covariance a bias E that bounds the rounding accumulated since the anchor:

    E = 2 eps C sqrt(N + 16),  eps = 2^-23,
    C = the largest, over the 512-row chunks since the anchor, of
        s_R s_C + 2 (df_R dg_C + df_C dg_R),

with s, df, dg the RMS over the chunk's rows (R) and over the columns it
stages (C: the chunk's rows shifted by the band's first diagonal, plus the
band width), and N the rows since the anchor.  Rounding errors of N steps add
up like a random walk, so E is a statistical bound (about five standard
deviations), not a worst case.  These tests emulate the recurrence in FP32
(a product of two FP32 values is exact in FP64, so FP64 add + one rounding
to FP32 is the fused multiply-add) against an FP64 recurrence, and check

* that E covers the error on random walks;
* that it must be the running maximum since the anchor: when the windows'
  norms drop (random walk, then white noise), the absolute error built up
  before the drop stays, and a bias from the current chunk alone is exceeded;
* that an anchor at the drop resets the error, so the bias there could be
  several times narrower;
* the same bound, plus its worst-case term for the rounding of h and of the
  score's two subtractions, on the non-normalised path;
* the FP32 anchors: the kernel starts each tile from an FP32 dot product of
  values centred in FP64 (the row window minus its mean; the column values
  minus one reference per block of diagonals, staged as FP32 hi + lo pairs
  and shifted in FP32 to a reference per 8 diagonals) and widens the bias to
  2 eps hypot(C sqrt(N + 16), B sqrt(m + 4)), B = ||a|| ||b|| the bound on
  the dot product's partial sums; emulated here step by step, from the FP32
  anchor against the exact FP64 walk, on random walks and on the same walks
  shifted by a large offset.
"""
import math

import numpy as np
import pytest

from paper_1904_12626_gb300 import synth

EPS32 = 2.0 ** -23
CHUNK = 512


def _stats(x, m):
    """mean, centred norm, df, dg per window (FP64, straightforward)."""
    l = len(x) - m + 1
    win = np.lib.stride_tricks.sliding_window_view(x, m)
    mu = win.mean(axis=1)
    s = np.linalg.norm(win - mu[:, None], axis=1)
    df = np.zeros(l)
    dg = np.zeros(l)
    df[1:] = (x[m:m + l - 1] - x[:l - 1]) / 2
    dg[1:] = (x[m:m + l - 1] - mu[1:]) + (x[:l - 1] - mu[:-1])
    return win, mu, s, df, dg


def _fma32(acc, x, y):
    """FP32 fused multiply-add, emulated: the product of two FP32 values is exact
    in FP64, and the sum is rounded once to FP32."""
    return np.float32(np.float64(acc) + np.float64(x) * np.float64(y))


def _anchor_f32(a, b, m, k0, width, d=8):
    """The kernel's FP32-mixed anchor at row 0 for diagonals k0..k0+width-1 of
    row series a against column series b: returns the FP32 covariances and B,
    the largest over the threads (d diagonals each) of ||a|| ||b_thread||."""
    f32 = np.float32
    mu_a = float(np.mean(a[:m]))
    mu_b = np.lib.stride_tricks.sliding_window_view(b, m).mean(axis=1)
    at = np.array([f32(v) for v in (a[:m] - mu_a)], dtype=np.float32)
    g0 = float(mu_b[k0 + width // 2])                   # the block's reference
    span = b[k0:k0 + width + m - 1].astype(np.float64) - g0
    hi = span.astype(np.float32)
    lo = (span - hi.astype(np.float64)).astype(np.float32)
    c = np.zeros(width, dtype=np.float32)
    bnd = 0.0
    for t0 in range(0, width, d):                       # one thread: d diagonals
        g = float(mu_b[k0 + t0 + d // 2]) - g0
        g_hi = f32(g)
        g_lo = f32(g - np.float64(g_hi))
        bv = ((hi[t0:t0 + m + d - 1] - g_hi).astype(np.float32)
              + (lo[t0:t0 + m + d - 1] - g_lo).astype(np.float32)).astype(np.float32)
        for dd in range(d):
            acc = f32(0.0)
            for t in range(m):
                acc = _fma32(acc, at[t], bv[dd + t])
            c[t0 + dd] = acc
        sa = float(np.sum(at.astype(np.float64) ** 2))
        sb = float(np.sum(bv.astype(np.float64) ** 2))
        bnd = max(bnd, math.sqrt(sa) * math.sqrt(sb))
    return c, bnd


def _walk(a, b, m, k0, width, rows, bias="running", anchor_rows=(), f32_anchor=False):
    """Walk diagonals k0..k0+width-1 (row i of a against column i+k of b) for
    `rows` rows from an anchor at row 0; returns the largest error / bias
    ratio per chunk, and the bias per chunk (correlation units of the
    chunk's first cell, for comparisons)."""
    winA, muA, sA, dfA, dgA = _stats(a, m)
    winB, muB, sB, dfB, dgB = _stats(b, m)
    ks = k0 + np.arange(width)

    def exact(i):
        return np.einsum("t,dt->d", winA[i] - muA[i], winB[i + ks] - muB[i + ks][:, None])

    f32 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    c64 = exact(0)
    c32 = c64.astype(np.float32)
    e_anchor = 0.0
    if f32_anchor:                                 # the kernel's FP32 anchor
        c32, bnd = _anchor_f32(a, b, m, k0, width)
        e_anchor = bnd * math.sqrt(m + 4)
    e_c, steps = 0.0, 0
    ratios, biases = [], []
    for r in range(0, rows, CHUNK):
        if r in anchor_rows:                       # exact covariance at row r - 1
            c64 = exact(r - 1)
            c32 = c64.astype(np.float32)
            e_c, steps = 0.0, 0
        R = slice(r, r + CHUNK)
        C = slice(r + k0, r + k0 + CHUNK + width)
        rms = lambda v: math.sqrt(float(np.mean(v * v)))
        cur = rms(sA[R]) * rms(sB[C]) + 2 * (rms(dfA[R]) * rms(dgB[C]) + rms(dfB[C]) * rms(dgA[R]))
        e_c = cur if bias == "current" else max(e_c, cur)
        steps += CHUNK
        E = 2.0 * EPS32 * math.hypot(e_c * math.sqrt(steps + 16), e_anchor)
        worst = 0.0
        if r == 0:                                 # the anchor itself
            worst = float(np.abs(c32.astype(np.float64) - c64).max()) / E
        for i in range(max(r, 1), r + CHUNK):
            j = i + ks
            c64 = c64 + dfA[i] * dgB[j] + dfB[j] * dgA[i]
            c32 = (c32.astype(np.float64) + f32(dfA[i]) * f32(dgB[j])).astype(np.float32)
            c32 = (c32.astype(np.float64) + f32(dfB[j]) * f32(dgA[i])).astype(np.float32)
            worst = max(worst, float(np.abs(c32.astype(np.float64) - c64).max()) / E)
        ratios.append(worst)
        biases.append(E / (sA[r] * sB[r + k0]))
    return np.array(ratios), np.array(biases)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bias_covers_fp32_rounding_on_random_walks(seed):
    m = 256
    a = synth.random_walk(12000, seed=seed)
    b = synth.random_walk(12000, seed=seed + 100)
    ratios, _ = _walk(a, b, m, k0=128, width=64, rows=8192)
    assert ratios.max() < 1.0
    assert ratios.max() > 0.02                     # and it is not vacuous


def _drop_input(seed, m):
    """rows: a random walk; columns: a random walk, then white noise (norm
    about 10x smaller) from sample 5000 on."""
    a = synth.random_walk(12000, seed=seed)
    rng = np.random.default_rng(seed + 7)
    b = np.concatenate([synth.random_walk(5000, seed=seed + 200), rng.standard_normal(7000)])
    return a, b


@pytest.mark.parametrize("seed", [0, 1])
def test_bias_must_be_the_running_maximum(seed):
    m = 256
    a, b = _drop_input(seed, m)
    running, _ = _walk(a, b, m, k0=0, width=64, rows=8192)
    current, _ = _walk(a, b, m, k0=0, width=64, rows=8192, bias="current")
    assert running.max() < 1.0
    assert current.max() > 1.5                     # after the drop the old error dominates
    assert current[:9].max() < 1.0                 # before it the two agree


def test_anchor_at_the_norm_drop_resets_the_error():
    m = 256
    a, b = _drop_input(0, m)
    drop = 5120                                    # first chunk whose columns are all white noise
    plain, bias_plain = _walk(a, b, m, k0=0, width=64, rows=8192)
    anchored, bias_anch = _walk(a, b, m, k0=0, width=64, rows=8192, anchor_rows=(drop,))
    after = slice(drop // CHUNK, None)
    assert anchored.max() < 1.0
    # the error-bias after the drop, in correlation units, is several times narrower
    assert np.median(bias_plain[after] / bias_anch[after]) > 5.0


def _walk_raw(x, m, k0, width, rows):
    """The non-normalised path (self-join): q(i,j) = sum x_i x_j walked with
    q += df_i dgr_j + df_j dgr_i (df = (x_{i+m-1} - x_{i-1}) / 2,
    dgr = x_{i+m-1} + x_{i-1}) in FP32, the score (q - h_j) - h_i with
    h = ||x_i||^2 / 2 rounded to FP32; the bias adds 4 eps (largest row h +
    largest column h) per chunk for the rounding of h and of the two
    subtractions.  Returns the largest |FP32 score - exact score| / E per chunk."""
    l = len(x) - m + 1
    win = np.lib.stride_tricks.sliding_window_view(x, m)
    h = 0.5 * np.einsum("it,it->i", win, win)
    df = np.zeros(l)
    dgr = np.zeros(l)
    df[1:] = (x[m:m + l - 1] - x[:l - 1]) / 2
    dgr[1:] = x[m:m + l - 1] + x[:l - 1]
    ks = k0 + np.arange(width)
    f32 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    q64 = np.einsum("t,dt->d", win[0], win[ks])
    q32 = q64.astype(np.float32)
    e_c, steps = 0.0, 0
    ratios = []
    rms = lambda v: math.sqrt(float(np.mean(v * v)))
    for r in range(0, rows, CHUNK):
        R = slice(r, r + CHUNK)
        C = slice(r + k0, r + k0 + CHUNK + width)
        e_c = max(e_c, math.sqrt(float(np.mean(2 * h[R]))) * math.sqrt(float(np.mean(2 * h[C])))
                  + 2 * (rms(df[R]) * rms(dgr[C]) + rms(df[C]) * rms(dgr[R])))
        steps += CHUNK
        E = 2.0 * EPS32 * (e_c * math.sqrt(steps + 16) + 2 * (h[R].max() + h[C].max()))
        worst = 0.0
        for i in range(max(r, 1), r + CHUNK):
            j = i + ks
            q64 = q64 + df[i] * dgr[j] + df[j] * dgr[i]
            q32 = (q32.astype(np.float64) + f32(df[i]) * f32(dgr[j])).astype(np.float32)
            q32 = (q32.astype(np.float64) + f32(df[j]) * f32(dgr[i])).astype(np.float32)
            score32 = (q32 - h[j].astype(np.float32)) - np.float32(h[i])
            exact = q64 - h[j] - h[i]
            worst = max(worst, float(np.abs(score32.astype(np.float64) - exact).max()) / E)
        ratios.append(worst)
    return np.array(ratios)


@pytest.mark.parametrize("seed", [0, 1])
def test_raw_bias_covers_fp32_rounding(seed):
    x = synth.tonal(12000, seed=seed)
    ratios = _walk_raw(x, 256, k0=128, width=64, rows=8192)
    assert ratios.max() < 1.0
    assert ratios.max() > 0.01


@pytest.mark.parametrize("seed,offset", [(0, 0.0), (1, 0.0), (2, 1.0e4)])
def test_bias_covers_fp32_anchor_and_recurrence(seed, offset):
    """From the FP32 anchor: the anchor's own error and the error after every
    chunk stay inside the widened bias, also when the series sit on a large
    offset (the centring is done in FP64, so the offset does not reach the
    FP32 sums)."""
    m = 256
    a = synth.random_walk(6000, seed=seed) + offset
    b = synth.random_walk(6000, seed=seed + 100) + offset
    ratios, _ = _walk(a, b, m, k0=128, width=32, rows=2048, f32_anchor=True)
    assert ratios.max() < 1.0
    assert ratios.max() > 0.02


def test_fp32_anchor_error_is_the_size_the_bias_allows():
    """The anchor's rounding is of the order of m recurrence steps: the FP32
    anchor's error alone is a visible fraction of the anchor term of the bias,
    2 eps B sqrt(m + 4), and well below it."""
    m = 512
    a = synth.random_walk(3000, seed=11)
    b = synth.random_walk(3000, seed=12)
    c32, bnd = _anchor_f32(a, b, m, k0=64, width=16)
    win_b = np.lib.stride_tricks.sliding_window_view(b, m)
    exact = np.array([np.dot(a[:m] - a[:m].mean(), win_b[64 + k] - win_b[64 + k].mean())
                      for k in range(16)])
    err = float(np.abs(c32.astype(np.float64) - exact).max())
    allowance = 2.0 * EPS32 * bnd * math.sqrt(m + 4)
    assert err < allowance
    assert err > 1e-3 * allowance
