"""GPU parity of the left / right self-join profiles (the profiles time series
chains are built on, Sec. 3.4.3): CUDA path through the C ABI vs the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

from _parity import check_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-3}


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    return api


def _run(mp, x, m, **kw):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return [t.cpu().numpy() for t in mp.selfjoin_lr(xt, m, check_status=True, **kw)]


def _check_sides(x, m, rows, g, o, tol, E, inclusive=False):
    gl, gpl, gr, gpr = g
    ml, pl, sl, mr, pr, sr = o
    check_rows(x, m, rows, gl, gpl, ml, pl, sl, tol, excl=E, inclusive=inclusive)
    check_rows(x, m, rows, gr, gpr, mr, pr, sr, tol, excl=E, inclusive=inclusive)
    # every reported neighbour lies on its side
    for i, j in zip(rows, gpl[rows]):
        assert j == -1 or j < i
    for i, j in zip(rows, gpr[rows]):
        assert j == -1 or j > i


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lr_random_walk_4096_all_rows(mp, prec):
    x = synth.random_walk(4096, seed=21)
    m = 64
    g = _run(mp, x, m, prec=prec)
    o = oracle.selfjoin_lr(x, m)
    _check_sides(x, m, np.arange(len(o[0])), g, o, TOL[prec], 32)
    # the two sides together give the self-join
    s_mp, s_pi = (t.cpu().numpy() for t in mp.selfjoin(torch.from_numpy(x).cuda(), m, prec=prec))
    np.testing.assert_array_equal(np.minimum(g[0], g[2]), s_mp)


@pytest.mark.parametrize("prec,variant", [("fp32", 0), ("fp32", 3), ("fp32", 4), ("fp64", 0)])
def test_lr_many_tiles_ragged(mp, prec, variant):
    x = synth.random_walk(3001, seed=22 + variant)
    m = 16
    g = _run(mp, x, m, prec=prec, variant=variant, tile_rows=300, anchor_every=128)
    o = oracle.selfjoin_lr(x, m)
    _check_sides(x, m, np.arange(len(o[0])), g, o, TOL[prec], 8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lr_edge_cases(mp, prec):
    # no admissible neighbour on either side
    x = synth.random_walk(20, seed=23)
    gl, gpl, gr, gpr = _run(mp, x, 16, prec=prec)
    assert np.isinf(gl).all() and np.isinf(gr).all() and (gpl == -1).all() and (gpr == -1).all()
    # flat stretch, inclusive zone, ez = 0.25
    x = synth.random_walk(1500, seed=24)
    x[200:260] = x[199]
    m = 32
    for ez, inclusive in ((0.5, False), (0.25, True)):
        E = oracle.exclusion_zone(m, ez)
        g = _run(mp, x, m, prec=prec, ez=ez, inclusive=inclusive)
        o = oracle.selfjoin_lr(x, m, ez, inclusive=inclusive)
        _check_sides(x, m, np.arange(len(o[0])), g, o, TOL[prec], E, inclusive)
        first = E + 1 if inclusive else E
        assert g[0][210] == math.sqrt(2 * m) and g[1][210] == 0          # flat: lowest left index
        assert g[2][210] == math.sqrt(2 * m) and g[3][210] == 210 + first  # lowest right index


def test_lr_near_flat_windows(mp):
    """Ill-conditioned windows go through the exact pass on each side."""
    x = synth.random_walk(12000, seed=25)
    x[3000:3400] = x[2999]
    x[3400:3404] = x[2999] + 1e-2 * np.array([1.0, -2.0, 3.0, 1.0])
    m = 128
    g = _run(mp, x, m, prec="fp32")
    rows = np.unique(np.concatenate([np.arange(2800, 3500), synth.sample_rows(len(x) - m + 1, 200,
                                                                             seed=26)]))
    o = oracle.selfjoin_lr(x, m, rows=rows)
    _check_sides(x, m, rows, g, o, TOL["fp32"], 64)


def test_lr_planted_full_size_sampled(mp):
    """n = 2^20 planted walk, m = 256 (the benchmark input), FP32-mixed."""
    n, m = 1 << 20, 256
    x, info = synth.planted_walk(n, m, seed=2024)
    g = _run(mp, x, m, prec="fp32")
    l = n - m + 1
    rows = np.unique(np.concatenate([synth.sample_rows(l, 96, seed=27),
                                     [p for pair in info["pairs"] for p in pair],
                                     [0, 1, 127, 128, l - 129, l - 128, l - 1]]))
    x64 = x.astype(np.float64)
    o = oracle.selfjoin_lr(x64, m, rows=rows)
    _check_sides(x64, m, rows, g, o, TOL["fp32"], 128)
    for p1, p2 in info["pairs"]:                 # a planted pair is each other's neighbour
        lo, hi = min(p1, p2), max(p1, p2)
        assert abs(g[3][lo] - hi) <= 2 and abs(g[1][hi] - lo) <= 2
