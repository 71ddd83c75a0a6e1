"""The device loops that retry are bounded and report when they run out.

Two loops may retry: the 128-bit compare-and-swap that merges an FP64-path
candidate into its key (at most kCasRetryLimit attempts), and the FP32-mixed
path's candidate merge (at most kMergeRounds rounds of decisions and exact
comparisons).  A loop that runs out records MP_ETIMEOUT in the workspace's
status word and returns; nothing waits.  The library's limits are far above
anything a join needs, so these tests build variants of the library (into a
temporary directory, leaving the package's own build alone) with one limit
set to 0 -- every merge that reaches the loop gives up at once -- run a small
join through the C ABI, and read the status word: the lowered loop reports
MP_ETIMEOUT, the other precision's join (which never enters it) reports
MP_OK, and in both cases the call came back.
"""
import ctypes

import numpy as np
import pytest

from paper_1904_12626_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _variant(tmp_path_factory, flag):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import _lib, build
    out = tmp_path_factory.mktemp("mpgb_" + flag.split("=")[0].lower().lstrip("-d"))
    path = build.build(extra_flags=(flag,), out_dir=str(out))
    lib = _lib.load(path)                  # a separate handle: the package's library is untouched
    assert lib.mp_init(torch.cuda.current_device()) == _lib.MP_OK
    return lib


@pytest.fixture(scope="module")
def no_cas_retries(tmp_path_factory):
    return _variant(tmp_path_factory, "-DMPGB_CAS_RETRY_LIMIT=0")


@pytest.fixture(scope="module")
def no_merge_rounds(tmp_path_factory):
    return _variant(tmp_path_factory, "-DMPGB_MERGE_ROUNDS=0")


def _selfjoin_status(lib, prec):
    """Status word after a self-join of a 6000-sample random walk (m = 64)."""
    from paper_1904_12626_gb300 import _lib
    n, m = 6000, 64
    x = torch.from_numpy(synth.random_walk(n, seed=91)).cuda()
    cfg = _lib.make_config(m, 0.5, prec)
    ws = torch.empty(lib.mp_selfjoin_workspace_bytes(n, ctypes.byref(cfg)), dtype=torch.uint8,
                     device="cuda")
    mp = torch.empty(n - m + 1, dtype=torch.float64, device="cuda")
    pi = torch.empty(n - m + 1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.mp_selfjoin(x.data_ptr(), _lib.MP_F64, n, ctypes.byref(cfg), mp.data_ptr(),
                           pi.data_ptr(), ws.data_ptr(), ws.numel(), st) == _lib.MP_OK
    code = lib.mp_get_device_status(ws.data_ptr(), st)        # synchronises: the join returned
    assert lib.mp_get_device_status(ws.data_ptr(), st) == _lib.MP_OK   # read and cleared
    return code


def test_cas_retry_limit_reports_timeout(no_cas_retries):
    from paper_1904_12626_gb300 import _lib
    assert _selfjoin_status(no_cas_retries, "fp64") == _lib.MP_ETIMEOUT
    assert _selfjoin_status(no_cas_retries, "fp32") == _lib.MP_OK


def test_merge_round_limit_reports_timeout(no_merge_rounds):
    from paper_1904_12626_gb300 import _lib
    assert _selfjoin_status(no_merge_rounds, "fp32") == _lib.MP_ETIMEOUT
    assert _selfjoin_status(no_merge_rounds, "fp64") == _lib.MP_OK


def test_default_limits_do_not_run_out():
    """The package's own build, on an input whose windows all have near-tied
    neighbours (a noisy sinusoid: every period is a near copy), finishes
    without a timeout and matches its FP64 twin's neighbours' distances."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    rng = np.random.default_rng(92)
    t = np.arange(8000)
    x = np.sin(2 * np.pi * t / 37.0) + 1e-3 * rng.standard_normal(len(t))
    xt = torch.from_numpy(x).cuda()
    a32, _ = api.selfjoin(xt, 64, 0.5, "fp32", check_status=True)
    a64, _ = api.selfjoin(xt, 64, 0.5, "fp64", check_status=True)
    assert float((a32 - a64).abs().max()) <= 1e-3
