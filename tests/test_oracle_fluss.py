"""Pins of the oracle's semantic segmentation (FLUSS, Sec. 3.4.2): a worked
example by hand, the O(l) arc count against the definition, the expected
arc count of random neighbours, and a regime change found by the oracle's own
self-join."""
import math

import numpy as np
import pytest

import oracle


def test_arc_counts_worked_example():
    # arcs: 0-2, 1-3, 2-0, 3-1; row 4 has no neighbour, row 5 points at itself
    pi = np.array([2, 3, 0, 1, -1, 5])
    # k=0: arcs 0-2 twice; k=1: 0-2 twice and 1-3 twice; k=2: 1-3 twice; k>=3: none
    expect = np.array([2, 4, 2, 0, 0, 0])
    np.testing.assert_array_equal(oracle.arc_counts(pi), expect)
    np.testing.assert_array_equal(oracle.arc_counts(pi, fast=True), expect)
    assert [oracle.arc_count_at(pi, k) for k in range(6)] == expect.tolist()
    cac, seg = oracle.fluss(pi, m=1, num_segments=2, edge=0, seg_excl=2)
    l = 6
    iac = np.array([2.0 * k * (l - k) / l for k in range(l)])
    want = np.ones(l)
    want[1:] = np.minimum(expect[1:] / iac[1:], 1.0)      # IAC[0] = 0 -> 1
    np.testing.assert_array_equal(cac, want)
    # lowest CAC: position 3 (0 arcs), then outside |k-3| < 2: positions 4, 5 are 0 too,
    # 4 is masked, 5 is the next lowest
    assert seg.tolist() == [3, 5]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fast_arc_counts_match_definition(seed):
    rng = np.random.default_rng(seed)
    l = 700
    pi = rng.integers(0, l, size=l)
    pi[rng.random(l) < 0.1] = -1
    pi[5] = 5
    np.testing.assert_array_equal(oracle.arc_counts(pi, fast=True), oracle.arc_counts(pi))


def test_random_neighbours_follow_the_idealised_curve():
    """Uniform random neighbours: E[AC[k]] = 2 (k+1)(l-k-1)/l, which is the
    idealised curve up to O(1); the mean ratio over the middle is 1."""
    rng = np.random.default_rng(7)
    l = 40000
    pi = rng.integers(0, l, size=l)
    ac = oracle.arc_counts(pi, fast=True)
    k = np.arange(l // 4, 3 * l // 4)
    iac = 2.0 * k * (l - k) / l
    ratio = ac[k] / iac
    assert abs(ratio.mean() - 1.0) < 0.01
    assert ratio.std() < 0.03


def test_edge_margin_by_hand():
    """One arc 0 -> 9 over l = 10 positions (AC = 1 on 0..8) with edge 2: the
    curve is 1 on the first and last two positions and AC / IAC on 2..7,
    IAC[k] = 2 k (l - k) / l."""
    pi = np.array([9, -1, -1, -1, -1, -1, -1, -1, -1, -1])
    cac, _ = oracle.fluss(pi, m=1, num_segments=0, edge=2, seg_excl=1)
    want = [1.0, 1.0, 1 / 3.2, 1 / 4.2, 1 / 4.8, 1 / 5.0, 1 / 4.8, 1 / 4.2, 1.0, 1.0]
    np.testing.assert_allclose(cac, want, rtol=1e-15)
    assert cac[2] < 1.0 and cac[7] < 1.0          # first and last positions outside the margin


def test_segment_masking():
    cac = np.array([0.9, 0.5, 0.4, 0.45, 0.9, 0.9, 0.2, 0.9, 0.3, 0.9])
    seg = np.empty(4, dtype=np.int64)
    lib = oracle.load()
    assert lib.oracle_segments(cac.ctypes.data_as(oracle._d), len(cac), 4, 2,
                               seg.ctypes.data_as(oracle._i64)) == 0
    # 6 (0.2); masked 5..7, the lowest left is 8 (0.3, |8-6| = 2 is outside);
    # masked 7..9, then 2 (0.4); masked 1..3, then 0 and 4 tie at 0.9: 0
    assert seg.tolist() == [6, 8, 2, 0]


def test_regime_change_found_by_selfjoin():
    """Two regimes (a sine, then a sawtooth of another period) with noise: the
    lowest corrected arc count sits at the change."""
    rng = np.random.default_rng(11)
    t = np.arange(3000)
    a = np.sin(2 * math.pi * t / 40.0)
    b = ((t % 25) / 25.0) * 2.0 - 1.0
    x = np.concatenate([a, b]) + 0.05 * rng.standard_normal(6000)
    m = 40
    mp, pi, _ = oracle.selfjoin(x, m)
    cac, seg = oracle.fluss(pi, m, num_segments=1)
    assert abs(int(seg[0]) - 3000) <= 2 * m
    assert cac[seg[0]] < 0.2
