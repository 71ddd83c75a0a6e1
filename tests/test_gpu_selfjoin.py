"""GPU parity of the self-join (CUDA path through the C ABI vs the CPU oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

import _golden
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
    a, b = mp.selfjoin(xt, m, check_status=True, **kw)
    return a.cpu().numpy(), b.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_random_walk_4096_all_rows(mp, prec):
    """n=4096 float64 random walk, m=64, E=32: every row against the oracle."""
    x = synth.random_walk(4096, seed=1)
    m = 64
    g_mp, g_pi = _run(mp, x, m, prec=prec)
    mp_o, pi_o, sec_o = oracle.selfjoin(x, m)
    rows = np.arange(len(mp_o))
    check_rows(x, m, rows, g_mp, g_pi, mp_o, pi_o, sec_o, TOL[prec], excl=32)


def test_fp32_without_refine(mp):
    x = synth.random_walk(4096, seed=2)
    m = 64
    g_mp, g_pi = _run(mp, x, m, prec="fp32", refine=False)
    mp_o, pi_o, sec_o = oracle.selfjoin(x, m)
    check_rows(x, m, np.arange(len(mp_o)), g_mp, g_pi, mp_o, pi_o, sec_o, 1e-3, excl=32)


@pytest.mark.parametrize("prec,variant", [("fp32", v) for v in range(8)] + [("fp64", v) for v in range(3)])
def test_variants_many_tiles_ragged(mp, prec, variant):
    """Small tiles so the matrix spans many bands and row tiles, with ragged
    tails on both axes; re-anchoring inside tiles."""
    from paper_1904_12626_gb300 import _lib
    assert variant < _lib.load().mp_variant_count(1 if prec == "fp32" else 0)
    x = synth.random_walk(3001, seed=3 + variant)
    m = 16
    g_mp, g_pi = _run(mp, x, m, prec=prec, variant=variant, tile_rows=300, anchor_every=128)
    mp_o, pi_o, sec_o = oracle.selfjoin(x, m)
    check_rows(x, m, np.arange(len(mp_o)), g_mp, g_pi, mp_o, pi_o, sec_o, TOL[prec], excl=8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_cases(mp, prec):
    tol = TOL[prec]
    # l = 1: no admissible neighbour
    x = synth.random_walk(40, seed=4)
    g_mp, g_pi = _run(mp, x, 40, prec=prec)
    assert np.isinf(g_mp).all() and (g_pi == -1).all()
    # l <= E: still nothing admissible
    x = synth.random_walk(20, seed=5)
    g_mp, g_pi = _run(mp, x, 16, prec=prec)
    assert np.isinf(g_mp).all() and (g_pi == -1).all()
    # smallest window, float32 input
    x = synth.random_walk(500, seed=6, dtype=np.float32)
    g_mp, g_pi = _run(mp, x, 4, prec=prec)
    mp_o, pi_o, sec_o = oracle.selfjoin(x.astype(np.float64), 4)
    check_rows(x.astype(np.float64), 4, np.arange(len(mp_o)), g_mp, g_pi, mp_o, pi_o, sec_o, tol,
               excl=2)
    # flat stretches, an exact scaled copy, other exclusion zones
    x = synth.random_walk(1500, seed=7)
    x[200:260] = x[199]
    x[900:932] = 3.5 * x[400:432] - 7.0
    for ez, inclusive in ((0.5, False), (0.25, False), (0.5, True), (1.0, False)):
        m = 32
        g_mp, g_pi = _run(mp, x, m, prec=prec, ez=ez, inclusive=inclusive)
        mp_o, pi_o, sec_o = oracle.selfjoin(x, m, ez, inclusive=inclusive)
        E = oracle.exclusion_zone(m, ez)
        check_rows(x, m, np.arange(len(mp_o)), g_mp, g_pi, mp_o, pi_o, sec_o, tol, excl=E,
                   inclusive=inclusive)
        assert g_mp[210] == math.sqrt(2 * m)                  # flat window: closed form
        assert g_mp[900] <= 1e-6 and g_pi[900] == 400          # exact copy
    # ez = 0: every window is its own neighbour
    x = synth.random_walk(300, seed=8)
    g_mp, g_pi = _run(mp, x, 16, prec=prec, ez=0.0)
    assert np.all(g_mp <= 1e-6) and np.array_equal(g_pi, np.arange(len(g_pi)))


@pytest.fixture(scope="module")
def planted():
    """The planted 2^20 walk and the oracle's answers on its sampled rows
    (4,096 seeded rows plus every planted row +-4)."""
    x, info, m = _golden.c2_inputs()
    answers, _ = _golden.c2_oracle(x, info, m)
    return x, info, m, answers


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_planted_full_size_sampled(mp, planted, prec):
    """n = 2^20 float32 random walk with 3 planted motif pairs and a planted
    discord, m = 256, in the launch configuration the benchmark times; the
    oracle checks 4,096 seeded rows plus every planted row +-4."""
    x, info, m, (rows, mp_o, pi_o, sec_o) = planted
    assert len(rows) >= 4096 + 60
    g_mp, g_pi = _run(mp, x, m, prec=prec)
    x64 = x.astype(np.float64)
    check_rows(x64, m, rows, g_mp, g_pi, mp_o, pi_o, sec_o, TOL[prec], excl=128)
    planted_rows = _golden.c2_planted_rows(info)
    assert np.isin(planted_rows, rows).all()
    for p1, p2 in info["pairs"]:
        assert abs(g_pi[p1] - p2) <= 2 and abs(g_pi[p2] - p1) <= 2
    top = int(np.argmax(g_mp))
    d = info["discord"]
    assert d - m + 1 <= top <= d + m - 1


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_near_flat_windows(mp, prec):
    """Windows that are constant except for a few small steps have norms
    thousands of times below the rest of the series; their correlations must
    still be exact.  The step patterns differ between the two stretches, so no
    two of these windows are exact copies (whose distance 0 would be decided
    by rounding alone)."""
    x = synth.random_walk(20000, seed=10)
    for s0, steps in ((3000, (1.0, -2.0, 3.0, 1.0)), (9000, (-2.0, 1.0, 1.0, -3.0))):
        x[s0:s0 + 400] = x[s0 - 1]
        x[s0 + 400:s0 + 404] = x[s0 - 1] + 1e-2 * np.array(steps)
    m = 128
    g_mp, g_pi = _run(mp, x, m, prec=prec)
    rows = np.unique(np.concatenate([np.arange(2800, 3700), np.arange(8800, 9700),
                                     synth.sample_rows(len(x) - m + 1, 300, seed=11)]))
    mp_o, pi_o, sec_o = oracle.selfjoin(x, m, rows=rows)
    check_rows(x, m, rows, g_mp, g_pi, mp_o, pi_o, sec_o, TOL[prec], excl=64)


def test_nonfinite_input_is_reported(mp):
    from paper_1904_12626_gb300 import _lib
    x = synth.random_walk(1000, seed=9)
    x[500] = np.nan
    with pytest.raises(_lib.MPError) as e:
        _run(mp, x, 32)
    assert e.value.code == _lib.MP_EINVAL_DATA
    # the workspace status was cleared: a clean call afterwards succeeds
    _run(mp, synth.random_walk(1000, seed=9), 32)
