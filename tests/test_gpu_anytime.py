"""GPU parity of the anytime self-join (random band order, partial runs,
resume; Sec. 3.3.1 / 3.3.3 and the s_size argument of Sec. 3.2) against the
oracle restricted to the diagonals each run has seen.

The band order is the library's documented generator, re-implemented here
from the published splitmix64 definition (Steele, Lea and Flood, 2014) and
the Fisher-Yates shuffle, so the test knows which diagonals a run covered."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

from _parity import check_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-3}
M64 = (1 << 64) - 1


def splitmix64_stream(seed):
    state = seed & M64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        yield z ^ (z >> 31)


def band_order(nb, seed):
    perm = list(range(nb))
    g = splitmix64_stream(seed)
    for i in range(nb - 1, 0, -1):
        j = next(g) % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def diag_mask(l, E, td, perm, s1):
    """Diagonals the first s1 slots cover, plus diagonal E (every key's seed)."""
    ok = np.zeros(l, bool)
    for b in perm[:s1]:
        lo = E + b * td
        ok[lo:min(lo + td, l)] = True
    if E < l:
        ok[E] = True
    return ok


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    return api


def _tile_diags(prec, variant):
    from paper_1904_12626_gb300 import _lib
    td, rc = ctypes.c_int32(), ctypes.c_int32()
    _lib.check(_lib.load().mp_variant_info(1 if prec == "fp32" else 0, variant, ctypes.byref(td),
                                           ctypes.byref(rc)), "variant info")
    return td.value


@pytest.mark.parametrize("prec,variant", [("fp32", 0), ("fp64", 0), ("fp32", 4)])
def test_anytime_partial_runs_and_resume(mp, prec, variant):
    n, m, seed = 6000, 32, 12345
    x = synth.random_walk(n, seed=41)
    l = n - m + 1
    E = oracle.exclusion_zone(m)
    td = _tile_diags(prec, variant)
    nb = (l - 1 - E) // td + 1
    perm = band_order(nb, seed)
    run = mp.Anytime(torch.from_numpy(x).cuda(), m, seed=seed, prec=prec, variant=variant)
    done = 0
    for f in (0.1, 0.35, 0.2, 0.7, 1.0):           # 0.2 after 0.35: nothing new
        g_mp, g_pi = (t.cpu().numpy() for t in run.run(f, check_status=True))
        done = max(done, math.ceil(f * nb))
        ok = diag_mask(l, E, td, perm, done)
        mo, po, so = oracle.selfjoin_diags(x, m, ok)
        rows = np.arange(l)
        check_rows(x, m, rows, g_mp, g_pi, mo, po, so, TOL[prec], excl=E)
        # every neighbour found lies on a covered diagonal
        has = g_pi >= 0
        assert ok[np.abs(g_pi[has] - rows[has])].all()
    s_mp, s_pi = (t.cpu().numpy() for t in mp.selfjoin(torch.from_numpy(x).cuda(), m, prec=prec,
                                                       variant=variant))
    np.testing.assert_array_equal(g_pi, s_pi)
    np.testing.assert_array_equal(g_mp, s_mp)


def test_anytime_seed_changes_order(mp):
    n, m = 6000, 32
    x = torch.from_numpy(synth.random_walk(n, seed=42)).cuda()
    a = mp.Anytime(x, m, seed=1).run(0.25)[0].cpu().numpy()
    b = mp.Anytime(x, m, seed=1).run(0.25)[0].cpu().numpy()
    c = mp.Anytime(x, m, seed=2).run(0.25)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert band_order(12, 1) != band_order(12, 2)


def test_anytime_full_size_five_percent(mp):
    """n = 2^20 planted walk, m = 256: a 5% run against the oracle over the
    same diagonals on sampled rows; the planted motif pairs' profile values
    can only improve as the run continues."""
    n, m, seed = 1 << 20, 256, 7
    x, info = synth.planted_walk(n, m, seed=2024)
    l = n - m + 1
    E = oracle.exclusion_zone(m)
    run = mp.Anytime(torch.from_numpy(x).cuda(), m, seed=seed)
    # the tile shape the library chose: the workspace header records its
    # diagonals per band (bytes 20..23)
    td = int(run.ws[20:24].cpu().numpy().view(np.int32)[0])
    assert td == _tile_diags("fp32", 7)
    nb = (l - 1 - E) // td + 1
    perm = band_order(nb, seed)
    g_mp, g_pi = (t.cpu().numpy() for t in run.run(0.05, check_status=True))
    ok = diag_mask(l, E, td, perm, math.ceil(0.05 * nb))
    rows = synth.sample_rows(l, 48, seed=43)
    x64 = x.astype(np.float64)
    mo, po, so = oracle.selfjoin_diags(x64, m, ok, rows=rows)
    check_rows(x64, m, rows, g_mp, g_pi, mo, po, so, TOL["fp32"], excl=E)
    g2, _ = (t.cpu().numpy() for t in run.run(0.5))
    assert np.all(g2 <= g_mp)
