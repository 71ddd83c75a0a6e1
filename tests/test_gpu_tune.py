"""The autotuner on the GPU: it times real candidates through the C ABI, the
configuration it picks reproduces the default configuration's result (the
FP32-mixed path certifies its neighbours, so exactly), that result matches
the oracle, and the choice is cached."""
import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

from _parity import check_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    return api


def test_tuned_selfjoin_equals_default_and_oracle(mp, tmp_path):
    from paper_1904_12626_gb300.tune import Tuner
    n, m = 40000, 64
    x_np = synth.random_walk(n, seed=91)
    x = torch.from_numpy(x_np).cuda()
    path = tmp_path / "tune.json"
    t = Tuner(path, warmup=1, reps=2)
    kw = t.selfjoin(x, m)
    ch = t.last
    assert set(kw) == {"variant", "tile_rows", "anchor_every"}
    assert ch.measured >= 8 and ch.ms <= ch.default_ms
    a, b = mp.selfjoin(x, m, check_status=True, **kw)
    a0, b0 = mp.selfjoin(x, m)
    assert torch.equal(a, a0) and torch.equal(b, b0)
    rows = synth.sample_rows(n - m + 1, 300, seed=92)
    mo, po, so = oracle.selfjoin(x_np, m, rows=rows)
    check_rows(x_np, m, rows, a.cpu().numpy(), b.cpu().numpy(), mo, po, so, 1e-3, excl=32)
    # the cached answer costs no measurement
    t2 = Tuner(path)
    assert t2.selfjoin(x, m) == kw and t2.measured == 0


@pytest.mark.parametrize("anchor_every", [512, 1024, 4096])
def test_anchor_interval_does_not_change_results(mp, anchor_every):
    """Every candidate the tuner can pick returns the same neighbours."""
    x = torch.from_numpy(synth.random_walk(30000, seed=93)).cuda()
    a0, b0 = mp.selfjoin(x, 128)
    for v in (0, 3):
        a, b = mp.selfjoin(x, 128, variant=v, tile_rows=8192, anchor_every=anchor_every,
                           check_status=True)
        assert torch.equal(a, a0) and torch.equal(b, b0)


def test_tuned_abjoin_fp64_within_budget(mp):
    from paper_1904_12626_gb300.tune import Tuner
    m = 48
    a_np = synth.random_walk(9000, seed=94)
    b_np = synth.random_walk(7000, seed=95)
    a, b = torch.from_numpy(a_np).cuda(), torch.from_numpy(b_np).cuda()
    kw = Tuner(None, warmup=0, reps=1).abjoin(a, b, m, "fp64")
    mpa, pia, mpb, pib = mp.abjoin(a, b, m, "fp64", check_status=True, **kw)
    rows = synth.sample_rows(len(a_np) - m + 1, 120, seed=96)
    mo, po, so = oracle.abjoin(a_np, b_np, m, rows=rows)
    check_rows(a_np, m, rows, mpa.cpu().numpy(), pia.cpu().numpy(), mo, po, so, 1e-9, y=b_np)


def test_tuned_batched_and_pan(mp):
    from paper_1904_12626_gb300.tune import Tuner
    t = Tuner(None, warmup=0, reps=1)
    values, offsets, ms = synth.ragged_batch(48, seed=97, len_lo=500, len_hi=3000)
    v = torch.from_numpy(values).cuda()
    o = torch.from_numpy(offsets).cuda()
    mm = torch.from_numpy(ms).cuda()
    kw = t.batched(v, o, mm)
    a, b, _ = mp.batched(v, o, mm, check_status=True, **kw)
    a0, b0, _ = mp.batched(v, o, mm)
    for s in range(len(ms)):
        lo, l_s = int(offsets[s]), int(offsets[s + 1] - offsets[s]) - int(ms[s]) + 1
        assert torch.equal(a[lo:lo + l_s], a0[lo:lo + l_s])
        assert torch.equal(b[lo:lo + l_s], b0[lo:lo + l_s])
    x = torch.from_numpy(synth.random_walk(6000, seed=98)).cuda()
    wins = [16, 40, 100]
    kw = t.pan(x, wins)
    p, q = mp.pan(x, wins, check_status=True, **kw)
    p0, q0 = mp.pan(x, wins)
    assert torch.equal(p, p0) and torch.equal(q, q0)
    assert len(t.entries) == 2
    assert np.isfinite(p.cpu().numpy()[0, :6000 - 16 + 1]).all()   # every window has a neighbour
