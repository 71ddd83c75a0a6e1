"""The bounds-checking build (-DMP_DEBUG) agrees with the release build.

Compiled with MP_DEBUG, the tile kernel and the exact pass for ill-conditioned
windows check every global index they compute from their descriptors -- the
staged rows and columns of statistics, the anchor row, the keys and thresholds
a candidate is merged into, the pairs compared exactly in FP64, the fragile
window of an exact-pass entry -- against the extent of the buffer it indexes.
An index outside it records MP_EBOUNDS in the workspace's status word and the
access is skipped.  These tests build that variant into a temporary directory
(the package's own library is untouched), swap it in as the binding's library,
run one small join of every family with the status checked, and compare the
results with the release build's: the checks must neither fire nor change an
answer.
"""
import numpy as np
import pytest

from paper_1904_12626_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import _lib, api, build
    build.build()
    api.init()
    path = build.build(extra_flags=("-DMP_DEBUG",), out_dir=str(tmp_path_factory.mktemp("mpgb_debug")))
    lib = _lib.load(path)                  # a separate handle: the package's library is untouched
    assert lib.mp_init(torch.cuda.current_device()) == _lib.MP_OK
    return lib


def _both(debug_lib, monkeypatch, fn):
    """fn() with the release library, then with the debug library."""
    from paper_1904_12626_gb300 import _lib
    rel = fn()
    with monkeypatch.context() as mc:
        mc.setattr(_lib, "_lib", debug_lib)
        dbg = fn()
    return rel, dbg


def _same(a, b):
    for u, v in zip(a, b):
        if u is None:
            assert v is None
            continue
        assert torch.equal(u.cpu(), v.cpu())


def _walk(n, seed):
    x = synth.random_walk(n, seed=seed)
    x[n // 3: n // 3 + 300] = x[n // 3]            # a flat stretch: ill-conditioned windows
    return torch.from_numpy(x).cuda()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_selfjoin_and_lr(debug_lib, monkeypatch, prec):
    from paper_1904_12626_gb300 import api
    x = _walk(20000, 301)
    rel, dbg = _both(debug_lib, monkeypatch, lambda: api.selfjoin(x, 128, 0.5, prec, check_status=True))
    _same(rel, dbg)
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.selfjoin_lr(x, 64, 0.5, prec, check_status=True))
    _same(rel, dbg)


def test_raw_and_anytime(debug_lib, monkeypatch):
    from paper_1904_12626_gb300 import api
    x = _walk(12000, 302)
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.selfjoin(x, 100, 0.5, "fp32", raw=True, check_status=True))
    _same(rel, dbg)
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.Anytime(x, 100, seed=7).run(0.3, check_status=True))
    _same(rel, dbg)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_abjoin(debug_lib, monkeypatch, prec):
    from paper_1904_12626_gb300 import api
    a, b = _walk(17000, 303), _walk(9001, 304)
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.abjoin(a, b, 96, prec, tile_rows=2048, check_status=True))
    _same(rel, dbg)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_and_pan(debug_lib, monkeypatch, prec):
    from paper_1904_12626_gb300 import api
    rng = np.random.default_rng(305)
    lens = rng.integers(200, 9000, size=24)
    vals = np.concatenate([synth.random_walk(int(k), seed=400 + i) for i, k in enumerate(lens)])
    offs = torch.tensor(np.concatenate([[0], np.cumsum(lens)]), dtype=torch.int64).cuda()
    ms = torch.tensor(rng.choice([16, 32, 64], size=len(lens)), dtype=torch.int32).cuda()
    v = torch.from_numpy(vals).cuda()
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.batched(v, offs, ms, 0.5, prec, check_status=True))
    # series b's profile is the first n_b - m_b + 1 of its n_b slots; the rest are unused
    used = np.concatenate([np.arange(o, o + k - mm + 1) for o, k, mm in
                           zip(offs.cpu().numpy()[:-1], lens, ms.cpu().numpy())])
    used = torch.from_numpy(used).cuda()
    _same([t[used] for t in rel[:2]], [t[used] for t in dbg[:2]])
    x = _walk(8000, 306)
    rel, dbg = _both(debug_lib, monkeypatch,
                     lambda: api.pan(x, [16, 40, 100, 257], 0.5, prec, check_status=True))
    _same(rel, dbg)
