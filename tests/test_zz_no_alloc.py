"""mp_selfjoin_noalloc: the self-join for callers that cannot allocate device
memory (inside someone else's graph capture, under an allocator that owns
all device memory, in a plugin given only its buffers).  It must give the
same profile as mp_selfjoin with a caller workspace, call after call, even
though every call reuses the library's one static scratch array.

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


def _noalloc(_lib, x, m, prec):
    lib = _lib.load()
    cfg = _lib.make_config(m, 0.5, prec)
    l = x.numel() - m + 1
    mp = torch.empty(l, dtype=torch.float64, device="cuda")
    pi = torch.empty(l, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib.mp_selfjoin_noalloc(x.data_ptr(), _lib.MP_F32 if x.dtype == torch.float32 else _lib.MP_F64,
                                       x.numel(), ctypes.byref(cfg), mp.data_ptr(), pi.data_ptr(), st),
               "mp_selfjoin_noalloc")
    return mp, pi


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-9)])
def test_matches_workspace_entry_point_twice(lib, prec, tol):
    from paper_1904_12626_gb300 import api
    # two calls in a row on different series: the second must not see the first's leftovers
    for n, m, seed in ((200_000, 128, 31), (150_001, 64, 32)):
        x = torch.from_numpy(synth.random_walk(n, seed=seed, dtype=np.float32)).cuda()
        mp_a, pi_a = _noalloc(lib, x, m, prec)
        mp_b, pi_b = api.selfjoin(x, m, 0.5, prec)
        torch.cuda.synchronize()
        assert torch.isfinite(mp_a).all()
        assert float((mp_a - mp_b).abs().max()) <= tol
        assert float((pi_a == pi_b).double().mean()) >= 0.999


def test_rejects_series_beyond_the_scratch(lib):
    cfg = lib.make_config(64)
    fake = 256 * 1024                      # rejected on the host before any use
    code = lib.load().mp_selfjoin_noalloc(fake, lib.MP_F32, 2_000_000, ctypes.byref(cfg), fake, fake, None)
    assert code == lib.MP_ENOMEM
