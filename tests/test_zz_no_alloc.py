"""mp_selfjoin_noalloc: the self-join for callers that cannot allocate device
memory (inside someone else's graph capture, under an allocator that owns
all device memory, in a plugin given only its buffers).  It must give the
same profile as mp_selfjoin with a caller workspace and the same
configuration -- bit for bit, call after call -- even though every call
reuses the library's one static scratch array.

Kept in a file pytest collects last so that a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1904_12626_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import _lib, api, build
    build.build()
    api.init()
    return _lib


def _dtype(lib, x):
    return lib.MP_F32 if x.dtype == torch.float32 else lib.MP_F64


def _noalloc(_lib, x, cfg):
    lib = _lib.load()
    l = x.numel() - cfg.m + 1
    mp = torch.empty(l, dtype=torch.float64, device="cuda")
    pi = torch.empty(l, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.mp_selfjoin_noalloc(x.data_ptr(), _dtype(_lib, x), x.numel(), ctypes.byref(cfg),
                                       mp.data_ptr(), pi.data_ptr(), st), "mp_selfjoin_noalloc")
    _lib.check(lib.mp_selfjoin_noalloc_device_status(st), "noalloc device status")
    return mp, pi


def _with_workspace(_lib, x, cfg):
    from paper_1904_12626_gb300 import api
    lib = _lib.load()
    l = x.numel() - cfg.m + 1
    mp = torch.empty(l, dtype=torch.float64, device="cuda")
    pi = torch.empty(l, dtype=torch.int64, device="cuda")
    ws = api.workspace(lib.mp_selfjoin_workspace_bytes(x.numel(), ctypes.byref(cfg)), x.device)
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.mp_selfjoin(x.data_ptr(), _dtype(_lib, x), x.numel(), ctypes.byref(cfg),
                               mp.data_ptr(), pi.data_ptr(), ws.data_ptr(), ws.numel(), st),
               "mp_selfjoin")
    api.device_status(ws)
    return mp, pi


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_matches_workspace_entry_point_twice(lib, prec):
    # two calls in a row on different series: the second must not see the
    # first's leftovers, and both equal the workspace entry point exactly
    for n, m, seed in ((200_000, 128, 31), (150_001, 64, 32)):
        x = torch.from_numpy(synth.random_walk(n, seed=seed, dtype=np.float32)).cuda()
        cfg = lib.make_config(m, 0.5, prec)
        mp_a, pi_a = _noalloc(lib, x, cfg)
        mp_b, pi_b = _with_workspace(lib, x, cfg)
        torch.cuda.synchronize()
        assert torch.isfinite(mp_a).all()
        assert torch.equal(mp_a, mp_b)
        assert torch.equal(pi_a, pi_b)


def test_size_limit(lib):
    """The largest n the scratch holds runs; one more sample is refused on the
    host before any work is enqueued."""
    l = lib.load()
    cfg = lib.make_config(64, 0.5, "fp32")
    n_max = l.mp_selfjoin_noalloc_max_n(ctypes.byref(cfg))
    assert n_max == 690_456                # the figure the header states
    assert l.mp_selfjoin_noalloc_max_n(ctypes.byref(lib.make_config(64, 0.5, "fp64"))) == 826_400
    x = torch.from_numpy(synth.random_walk(n_max, seed=33, dtype=np.float32)).cuda()
    mp_a, pi_a = _noalloc(lib, x, cfg)
    assert torch.isfinite(mp_a).all() and (pi_a >= 0).all()
    fake = 256 * 1024                      # never dereferenced: rejected on the host
    code = l.mp_selfjoin_noalloc(fake, lib.MP_F32, n_max + 1, ctypes.byref(cfg), fake, fake, None)
    assert code == lib.MP_ENOMEM


def test_device_status_is_readable(lib):
    """A non-finite input is reported through the scratch's status word, which
    the getter clears; the next clean call then reports nothing."""
    l = lib.load()
    cfg = lib.make_config(32, 0.5, "fp32")
    x = synth.random_walk(5000, seed=34, dtype=np.float32)
    x[1234] = np.nan
    xt = torch.from_numpy(x).cuda()
    mp = torch.empty(5000 - 31, dtype=torch.float64, device="cuda")
    pi = torch.empty(5000 - 31, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert l.mp_selfjoin_noalloc(xt.data_ptr(), lib.MP_F32, 5000, ctypes.byref(cfg), mp.data_ptr(),
                                 pi.data_ptr(), st) == lib.MP_OK
    assert l.mp_selfjoin_noalloc_device_status(st) == lib.MP_EINVAL_DATA
    assert l.mp_selfjoin_noalloc_device_status(st) == lib.MP_OK
    x[1234] = 0.0
    _noalloc(lib, torch.from_numpy(x).cuda(), cfg)
