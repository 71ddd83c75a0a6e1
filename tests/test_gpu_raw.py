"""GPU parity of the non-normalised distance (SiMPle's ||x_i - x_j||, no
z-normalisation, Sec. 3.3.4; MP_FLAG_RAW) against the oracle's brute force."""
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["tonal", "walk"])
def test_raw_selfjoin_all_rows(mp, prec, kind):
    x = synth.tonal(4096, seed=61) if kind == "tonal" else synth.random_walk(4096, seed=62)
    x[1000:1100] = x[999]                       # a flat stretch: ordinary windows here
    m = 64
    g_mp, g_pi = (t.cpu().numpy() for t in mp.selfjoin(_t(x), m, prec=prec, raw=True,
                                                       check_status=True))
    mo, po, so = oracle.join_raw(x, m)
    check_rows(x, m, np.arange(len(mo)), g_mp, g_pi, mo, po, so, TOL[prec], excl=32, raw=True)


def test_raw_many_tiles_ragged(mp):
    x = synth.tonal(3001, seed=63)
    m = 16
    for prec in ("fp32", "fp64"):
        g_mp, g_pi = (t.cpu().numpy() for t in mp.selfjoin(_t(x), m, prec=prec, raw=True,
                                                           tile_rows=300, anchor_every=128))
        mo, po, so = oracle.join_raw(x, m)
        check_rows(x, m, np.arange(len(mo)), g_mp, g_pi, mo, po, so, TOL[prec], excl=8, raw=True)


def test_raw_abjoin_and_sides(mp):
    a = synth.tonal(1 << 16, seed=64, dtype=np.float32)
    b = synth.tonal(1 << 15, seed=65, dtype=np.float32)
    m = 128
    ma, pa, mb, pb = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec="fp32", raw=True,
                                                         check_status=True))
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    rows = synth.sample_rows(len(a) - m + 1, 64, seed=66)
    mo, po, so = oracle.join_raw(a64, m, b=b64, rows=rows)
    check_rows(a64, m, rows, ma, pa, mo, po, so, TOL["fp32"], y=b64, raw=True)
    rows = synth.sample_rows(len(b) - m + 1, 64, seed=67)
    mo, po, so = oracle.join_raw(b64, m, b=a64, rows=rows)
    check_rows(b64, m, rows, mb, pb, mo, po, so, TOL["fp32"], y=a64, raw=True)
    # left/right sides with the raw distance combine to the raw self-join
    x = synth.tonal(5000, seed=68)
    gl, gpl, gr, gpr = (t.cpu().numpy() for t in mp.selfjoin_lr(_t(x), 32, prec="fp64", raw=True))
    s_mp, _ = (t.cpu().numpy() for t in mp.selfjoin(_t(x), 32, prec="fp64", raw=True))
    np.testing.assert_array_equal(np.minimum(gl, gr), s_mp)


def test_raw_full_size_sampled(mp):
    """n = 2^20 tonal signal, m = 256, FP32-mixed, sampled rows."""
    n, m = 1 << 20, 256
    x = synth.tonal(n, seed=69, dtype=np.float32)
    g_mp, g_pi = (t.cpu().numpy() for t in mp.selfjoin(_t(x), m, prec="fp32", raw=True,
                                                       check_status=True))
    rows = synth.sample_rows(n - m + 1, 48, seed=70)
    x64 = x.astype(np.float64)
    mo, po, so = oracle.join_raw(x64, m, rows=rows)
    check_rows(x64, m, rows, g_mp, g_pi, mo, po, so, TOL["fp32"], excl=128, raw=True)


def test_raw_needs_variant_zero(mp):
    """The non-normalised kernels exist in the default shape only: another
    variant is refused by the workspace query (0 bytes) and the call."""
    import ctypes

    from paper_1904_12626_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.make_config(32, 0.5, "fp32", 0, 0, 1, _lib.MP_FLAG_RAW)
    assert lib.mp_selfjoin_workspace_bytes(1000, ctypes.byref(cfg)) == 0
    x = _t(synth.tonal(1000, seed=71))
    out = torch.empty(1000, dtype=torch.float64, device="cuda")
    idx = torch.empty(1000, dtype=torch.int64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    rc = lib.mp_selfjoin(x.data_ptr(), _lib.MP_F64, 1000, ctypes.byref(cfg), out.data_ptr(),
                         idx.data_ptr(), ws.data_ptr(), ws.numel(), None)
    assert rc == _lib.MP_EUNSUPPORTED
