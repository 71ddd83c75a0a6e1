"""Pins for the CPU oracle, checked against what the definition and the paper
fix, never against the oracle's own formulas:

* the paper's printed profile sizes and exclusion zones (Sec. 3.2, 3.4);
* the Pearson identity d^2 = 2m(1 - rho), rho from numpy.corrcoef;
* bounds, affine-copy invariance, symmetry and the flat-window convention;
* brute force on small inputs through scipy (zscore + cdist);
* planted motif pairs and a planted discord (the MP properties of Sec. 2);
* the diagonal-recurrence identity on exact integer data;
* the closed-form gradient against central finite differences.
"""
import math
import os
import warnings

import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view

import oracle
from paper_1904_12626_gb300 import synth

scipy_stats = pytest.importorskip("scipy.stats")
scipy_dist = pytest.importorskip("scipy.spatial.distance")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_sizes.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, w, ez, l, e = line.split()[:5]
            rows.append((None if n == "-" else int(n), int(w), float(ez),
                         None if l == "-" else int(l), int(e)))
    return rows


def test_paper_printed_sizes():
    rows = _golden_rows()
    assert len(rows) == 4
    for n, w, ez, l, e in rows:
        if n is not None:
            assert oracle.profile_length(n, w) == l
        assert oracle.exclusion_zone(w, ez) == e
    # 50 * 1/4 = 12.5 must round up (13), not to even (12)
    assert oracle.exclusion_zone(50, 0.25) == 13


def _scipy_profile(x, m, excl=None, inclusive=False, y=None, side=0, diag_ok=None):
    """MP/PI by scipy: z-normalise every window (population std), full
    Euclidean distance matrix, mask, row minimum.  Flat windows follow the
    stated convention (distance sqrt(2m) to everything).  side = -1 / +1
    keeps only the candidates before / after each row."""
    wa = sliding_window_view(np.asarray(x, np.float64), m)
    wb = wa if y is None else sliding_window_view(np.asarray(y, np.float64), m)
    flat_a = np.ptp(wa, axis=1) == 0
    flat_b = np.ptp(wb, axis=1) == 0
    with np.errstate(invalid="ignore", divide="ignore"), warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)   # flat windows: 0/0
        za = scipy_stats.zscore(wa, axis=1, ddof=0)
        zb = scipy_stats.zscore(wb, axis=1, ddof=0)
    za[flat_a] = 0.0
    zb[flat_b] = 0.0
    D = scipy_dist.cdist(za, zb, "euclidean")
    D[flat_a, :] = math.sqrt(2 * m)
    D[:, flat_b] = math.sqrt(2 * m)
    D = np.minimum(D, 2 * math.sqrt(m))
    if excl is not None:
        ii, jj = np.indices(D.shape)
        bad = np.abs(ii - jj) <= excl if inclusive else np.abs(ii - jj) < excl
        if side < 0:
            bad |= jj >= ii
        elif side > 0:
            bad |= jj <= ii
        if diag_ok is not None:
            bad |= ~np.asarray(diag_ok, bool)[np.abs(ii - jj)]
        D[bad] = np.inf
    pi = np.argmin(D, axis=1)
    mp = D[np.arange(len(D)), pi]
    pi = np.where(np.isinf(mp), -1, pi)
    srt = np.sort(D, axis=1)
    with np.errstate(invalid="ignore"):            # inf - inf where a row has no neighbour
        gap = srt[:, 1] - srt[:, 0] if D.shape[1] > 1 else np.full(len(D), np.inf)
    return mp, pi, gap


def test_window_stats_against_numpy():
    x = synth.random_walk(700, seed=3)
    for m in (4, 17, 64):
        mu, sig, flat = oracle.window_stats(x, m)
        w = sliding_window_view(x, m)
        np.testing.assert_allclose(mu, w.mean(axis=1), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(sig, w.std(axis=1), rtol=1e-12, atol=1e-12)
        assert not flat.any()


def test_distance_is_pearson_identity():
    """d^2 = 2m(1 - rho) with rho from numpy's Pearson correlation."""
    rng = np.random.default_rng(11)
    x = synth.random_walk(3000, seed=5)
    for m in (8, 50, 256):
        l = len(x) - m + 1
        for _ in range(40):
            i, j = (int(v) for v in rng.integers(0, l, 2))
            rho = np.corrcoef(x[i:i + m], x[j:j + m])[0, 1]
            d = oracle.distance(x, m, i, j)
            expect = math.sqrt(max(0.0, 2 * m * (1 - rho)))
            assert abs(d - expect) <= 1e-9 * max(1.0, expect)
            assert 0.0 <= d <= 2 * math.sqrt(m) + 1e-12


def test_affine_copy_invariance():
    rng = np.random.default_rng(2)
    m = 64
    x = synth.random_walk(1000, seed=8)
    i, j = 100, 600
    for a, b in ((3.7, -50.0), (1e-3, 1e4), (250.0, 0.25)):
        y = x.copy()
        y[j:j + m] = a * x[i:i + m] + b
        # the copy itself is rounded to FP64: allow that input error, scaled
        # by the window's spread (8 sqrt(m) ulps of the copied values)
        slack = 8 * math.sqrt(m) * np.finfo(float).eps * np.abs(y[j:j + m]).max() / np.std(y[j:j + m])
        assert oracle.distance(y, m, i, j) <= 1e-9 + slack
    y = x.copy()
    y[j:j + m] = -2.5 * x[i:i + m] + rng.normal()
    assert abs(oracle.distance(y, m, i, j) - 2 * math.sqrt(m)) <= 1e-9


def test_distance_never_exceeds_the_bound():
    """A negated copy is at distance 2 sqrt(m) exactly in exact arithmetic;
    rounding may land just above, and the convention clamps d to [0, 2 sqrt(m)]
    with no slack (20 seeded windows of random length, scale and offset: in
    about half of them the unclamped FP64 value exceeds the bound)."""
    for seed in range(20):
        rng = np.random.default_rng(seed)
        m = int(rng.integers(8, 300))
        w = rng.standard_normal(m) * rng.uniform(0.1, 10) + rng.uniform(-100, 100)
        x = np.concatenate([w, -w])
        d = oracle.distance(x, m, 0, m)
        assert d <= 2 * math.sqrt(m)
        assert d >= 2 * math.sqrt(m) - 1e-9


def test_distance_symmetry_bitwise():
    x = synth.random_walk(900, seed=21)
    a = synth.random_walk(400, seed=22)
    rng = np.random.default_rng(1)
    m = 32
    for _ in range(50):
        i, j = (int(v) for v in rng.integers(0, len(x) - m + 1, 2))
        assert oracle.distance(x, m, i, j) == oracle.distance(x, m, j, i)
        ia = int(rng.integers(0, len(a) - m + 1))
        assert oracle.distance_ab(a, x, m, ia, j) == oracle.distance_ab(x, a, m, j, ia)


def test_flat_convention():
    m = 16
    x = synth.random_walk(300, seed=4)
    x[100:140] = x[99]            # windows 99..124 are flat
    mu, sig, flat = oracle.window_stats(x, m)
    w = sliding_window_view(x, m)
    np.testing.assert_array_equal(flat, np.ptp(w, axis=1) == 0)
    assert flat[99] and flat[124] and not flat[125] and not flat[98]
    s2m = math.sqrt(2 * m)
    assert oracle.distance(x, m, 110, 10) == s2m
    assert oracle.distance(x, m, 10, 110) == s2m
    assert oracle.distance(x, m, 105, 120) == s2m
    mp, pi, _ = oracle.selfjoin(x, m, rows=[110])
    assert mp[0] == s2m and pi[0] == 0        # everything ties; lowest index wins


@pytest.mark.parametrize("n,m,ez,inclusive,seed", [
    (64, 8, 0.5, False, 1), (64, 8, 0.5, True, 2), (200, 12, 0.25, False, 3),
    (301, 16, 0.5, False, 4), (150, 4, 1.0, False, 5)])
def test_selfjoin_against_scipy_bruteforce(n, m, ez, inclusive, seed):
    x = synth.random_walk(n, seed=seed)
    if seed == 4:
        x[40:70] = x[39]                      # include flat windows
    E = oracle.exclusion_zone(m, ez)
    mp, pi, sec = oracle.selfjoin(x, m, ez, inclusive=inclusive)
    mp_s, pi_s, gap = _scipy_profile(x, m, E, inclusive)
    np.testing.assert_allclose(mp, mp_s, rtol=0, atol=1e-10)
    sep = gap > 1e-9
    np.testing.assert_array_equal(pi[sep], pi_s[sep])
    np.testing.assert_allclose((sec - mp)[sep], gap[sep], atol=1e-9)


@pytest.mark.parametrize("n,m,ez,inclusive,seed", [
    (64, 8, 0.5, False, 11), (120, 8, 0.25, True, 12), (301, 16, 0.5, False, 13)])
def test_selfjoin_lr_against_scipy_bruteforce(n, m, ez, inclusive, seed):
    """Left / right profiles (the basis of time series chains, Sec. 3.4.3):
    the self-join definition with the candidates cut at the row."""
    x = synth.random_walk(n, seed=seed)
    if seed == 13:
        x[40:70] = x[39]                      # flat windows on both sides
    E = oracle.exclusion_zone(m, ez)
    ml, pl, sl, mr, pr, sr = oracle.selfjoin_lr(x, m, ez, inclusive=inclusive)
    for side, mp, pi, sec in ((-1, ml, pl, sl), (1, mr, pr, sr)):
        mp_s, pi_s, gap = _scipy_profile(x, m, E, inclusive, side=side)
        np.testing.assert_array_equal(np.isinf(mp), np.isinf(mp_s))
        fin = np.isfinite(mp_s)
        np.testing.assert_allclose(mp[fin], mp_s[fin], rtol=0, atol=1e-10)
        np.testing.assert_array_equal(pi[~fin], -1)
        sep = fin & (gap > 1e-9)
        np.testing.assert_array_equal(pi[sep], pi_s[sep])
    # no left neighbour for the first E rows, no right one for the last E
    first = E + 1 if inclusive else E
    assert np.all(np.isinf(ml[:first])) and np.all(np.isfinite(ml[first:]))
    assert np.all(np.isinf(mr[-first:])) and np.all(np.isfinite(mr[:-first]))
    # the two sides together are the self-join
    mp, pi, _ = oracle.selfjoin(x, m, ez, inclusive=inclusive)
    np.testing.assert_array_equal(np.minimum(ml, mr), mp)
    take_left = ml <= mr
    np.testing.assert_array_equal(np.where(take_left, pl, pr), pi)


def test_selfjoin_diags_against_scipy_and_special_cases():
    """An anytime run's best-so-far over a set of diagonals (Sec. 3.3.1,
    3.3.3): scipy with the same mask; every diagonal allowed is the self-join;
    one diagonal k gives min(d(i, i+k), d(i, i-k))."""
    x = synth.random_walk(260, seed=17)
    m = 8
    l = len(x) - m + 1
    E = oracle.exclusion_zone(m)
    rng = np.random.default_rng(18)
    ok = rng.random(l) < 0.3
    mp, pi, _ = oracle.selfjoin_diags(x, m, ok)
    mp_s, pi_s, gap = _scipy_profile(x, m, E, diag_ok=ok)
    np.testing.assert_array_equal(np.isinf(mp), np.isinf(mp_s))
    fin = np.isfinite(mp_s)
    np.testing.assert_allclose(mp[fin], mp_s[fin], atol=1e-10)
    sep = fin & (gap > 1e-9)
    np.testing.assert_array_equal(pi[sep], pi_s[sep])
    full = oracle.selfjoin(x, m)
    allm = oracle.selfjoin_diags(x, m, np.ones(l, bool))
    np.testing.assert_array_equal(allm[0], full[0])
    np.testing.assert_array_equal(allm[1], full[1])
    k = 37
    one = np.zeros(l, bool)
    one[k] = True
    mp1, pi1, _ = oracle.selfjoin_diags(x, m, one)
    for i in range(l):
        cands = [j for j in (i - k, i + k) if 0 <= j < l]
        ds = [oracle.distance(x, m, i, j) for j in cands]
        assert mp1[i] == min(ds) and pi1[i] == cands[int(np.argmin(ds))]


@pytest.mark.parametrize("inclusive", [False, True])
def test_raw_join_against_scipy(inclusive):
    """Non-normalised distance (SiMPle, Sec. 3.3.4): scipy's Euclidean
    distance matrix of the raw windows; shift and scale behave as the
    definition says; flat windows get no special rule."""
    rng = np.random.default_rng(19)
    x = np.cumsum(rng.standard_normal(240))
    x[60:90] = x[59]                          # flat windows are ordinary here
    m = 10
    E = oracle.exclusion_zone(m)
    W = sliding_window_view(x, m)
    D = scipy_dist.cdist(W, W, "euclidean")
    ii, jj = np.indices(D.shape)
    D[(np.abs(ii - jj) <= E) if inclusive else (np.abs(ii - jj) < E)] = np.inf
    mp, pi, _ = oracle.join_raw(x, m, inclusive=inclusive)
    np.testing.assert_allclose(mp, D.min(axis=1), atol=1e-10)
    srt = np.sort(D, axis=1)
    sep = srt[:, 1] - srt[:, 0] > 1e-9
    np.testing.assert_array_equal(pi[sep], D.argmin(axis=1)[sep])
    mp2, pi2, _ = oracle.join_raw(3.0 * x - 11.0, m, inclusive=inclusive)
    np.testing.assert_allclose(mp2, 3.0 * mp, rtol=1e-9)
    np.testing.assert_array_equal(pi2[sep], pi[sep])
    b = rng.standard_normal(150)
    mpab, piab, _ = oracle.join_raw(x, m, b=b)
    Dab = scipy_dist.cdist(W, sliding_window_view(b, m), "euclidean")
    np.testing.assert_allclose(mpab, Dab.min(axis=1), atol=1e-10)
    np.testing.assert_array_equal(piab, Dab.argmin(axis=1))


def test_abjoin_against_scipy_bruteforce():
    a = synth.random_walk(180, seed=7)
    b, _ = synth.mixed_with_flats(260, 8, seed=9, block=32, n_flat=2, flat_len=16)
    m = 8
    mp, pi, _ = oracle.abjoin(a, b, m)
    mp_s, pi_s, gap = _scipy_profile(a, m, None, y=b)
    np.testing.assert_allclose(mp, mp_s, atol=1e-10)
    sep = gap > 1e-9
    np.testing.assert_array_equal(pi[sep], pi_s[sep])
    # join symmetry: B's nearest in A equals the BA-join's A-side answer
    mp_b, pi_b, _ = oracle.abjoin(b, a, m)
    mp_bs, pi_bs, gap_b = _scipy_profile(b, m, None, y=a)
    np.testing.assert_allclose(mp_b, mp_bs, atol=1e-10)
    np.testing.assert_array_equal(pi_b[gap_b > 1e-9], pi_bs[gap_b > 1e-9])


def test_no_admissible_neighbour():
    x = synth.random_walk(20, seed=1)
    m = 16                                     # l = 5, E = 8: nothing admissible
    mp, pi, _ = oracle.selfjoin(x, m)
    assert np.all(np.isinf(mp)) and np.all(pi == -1)


def test_planted_motifs_and_discord():
    m = 64
    x, info = synth.planted_walk(3000, m, seed=12, n_pairs=3, dtype=np.float64)
    mp, pi, _ = oracle.selfjoin(x, m)
    near_planted = np.zeros(len(mp), bool)
    for p1, p2 in info["pairs"]:
        assert abs(pi[p1] - p2) <= 2 and abs(pi[p2] - p1) <= 2
        near_planted[max(0, p1 - m):p1 + m] = True
        near_planted[max(0, p2 - m):p2 + m] = True
    d = info["discord"]
    near_planted[max(0, d - m):d + m] = True
    for p1, p2 in info["pairs"]:
        assert max(mp[p1], mp[p2]) < mp[~near_planted].min()
    top = int(np.argmax(mp))
    assert d - m + 1 <= top <= d + m - 1


def test_recurrence_identity_exact_on_integers():
    """c(i,j) - c(i-1,j-1) = df_i dg_j + df_j dg_i, exactly on small integer
    data with a power-of-two window (every intermediate is a dyadic rational
    FP64 holds exactly); and the recurrence run from c(0,k) reproduces the
    direct c(i,i+k) exactly."""
    rng = np.random.default_rng(5)
    x = rng.integers(-20, 21, size=200).astype(np.float64)
    m = 16
    df, dg = oracle.mpx_terms(x, m)
    l = len(x) - m + 1
    for _ in range(200):
        i = int(rng.integers(1, l))
        j = int(rng.integers(1, l))
        lhs = oracle.cov(x, x, m, i, j) - oracle.cov(x, x, m, i - 1, j - 1)
        assert lhs == df[i] * dg[j] + df[j] * dg[i]
    for k in (8, 30, 111):
        c = oracle.cov(x, x, m, 0, k)
        for i in range(1, l - k):
            c = c + df[i] * dg[i + k] + df[i + k] * dg[i]
            assert c == oracle.cov(x, x, m, i, i + k)


def test_recurrence_identity_cross_series():
    a = synth.random_walk(300, seed=30)
    b = synth.random_walk(250, seed=31)
    m = 24
    dfa, dga = oracle.mpx_terms(a, m)
    dfb, dgb = oracle.mpx_terms(b, m)
    rng = np.random.default_rng(3)
    for _ in range(100):
        i = int(rng.integers(1, len(a) - m + 1))
        j = int(rng.integers(1, len(b) - m + 1))
        lhs = oracle.cov(a, b, m, i, j) - oracle.cov(a, b, m, i - 1, j - 1)
        rhs = dfa[i] * dgb[j] + dfb[j] * dga[i]
        assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def _mp_full(x, m):
    mp, pi, _ = oracle.selfjoin(x, m)
    return mp, pi


def test_gradient_against_central_differences():
    n, m, h = 200, 12, 1e-6
    x = synth.random_walk(n, seed=44)
    mp, pi = _mp_full(x, m)
    g = np.ones_like(mp)
    g[np.argsort(-mp, kind="stable")[:8]] += 1.0 / 8
    grad = oracle.grad(x, m, pi, g)
    fd = np.empty(n)
    keep = np.ones(n, bool)
    for p in range(n):
        xp, xm = x.copy(), x.copy()
        xp[p] += h
        xm[p] -= h
        mpp, pip = _mp_full(xp, m)
        mpm, pim = _mp_full(xm, m)
        if not (np.array_equal(pip, pi) and np.array_equal(pim, pi)):
            keep[p] = False                    # an argmin flips: not differentiable here
            continue
        fd[p] = (np.dot(g, mpp) - np.dot(g, mpm)) / (2 * h)
    assert keep.mean() > 0.8
    err = np.linalg.norm(grad[keep] - fd[keep]) / np.linalg.norm(fd[keep])
    assert err <= 1e-5
