"""Host-side checks of the C ABI: the library builds, loads on a machine
without a GPU, exports every entry point include/mp.h declares, and its
host helpers and argument checks behave (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1904_12626_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mp.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in mp.h but not exported"
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_paper_sizes_through_the_abi(lib):
    golden = os.path.join(ROOT, "tests", "golden", "paper_worked_sizes.txt")
    for line in open(golden):
        if line.startswith("#") or not line.strip():
            continue
        n, w, ez, l, e = line.split()[:5]
        if n != "-":
            assert lib.mp_profile_length(int(n), int(w)) == int(l)
        assert lib.mp_exclusion_zone(int(w), float(ez)) == int(e)
    assert lib.mp_profile_length(10, 11) == 0


def test_config_defaults_and_variants(lib):
    cfg = _lib.MPConfig()
    lib.mp_config_default(ctypes.byref(cfg), 256)
    assert cfg.m == 256 and cfg.ez == 0.5 and cfg.prec == _lib.MP_PREC_FP32_MIXED and cfg.flags == 0
    for prec in (_lib.MP_PREC_FP32_MIXED, _lib.MP_PREC_FP64):
        nv = lib.mp_variant_count(prec)
        assert nv >= 2
        for v in range(nv):
            td, rc = ctypes.c_int32(), ctypes.c_int32()
            assert lib.mp_variant_info(prec, v, ctypes.byref(td), ctypes.byref(rc)) == 0
            assert td.value % 32 == 0 and 0 < td.value <= 1024 and rc.value > 0
        assert lib.mp_variant_info(prec, nv, None, None) == _lib.MP_EINVAL
    assert lib.mp_version().decode().startswith("mpgb")


def test_workspace_sizes(lib):
    cfg = _lib.make_config(256)
    a = lib.mp_selfjoin_workspace_bytes(1 << 16, ctypes.byref(cfg))
    b = lib.mp_selfjoin_workspace_bytes(1 << 20, ctypes.byref(cfg))
    assert 0 < a < b and a % 256 == 0
    cfg64 = _lib.make_config(256, prec="fp64")
    assert lib.mp_selfjoin_workspace_bytes(1 << 20, ctypes.byref(cfg64)) > 0
    assert lib.mp_abjoin_workspace_bytes(1 << 21, 1 << 19, ctypes.byref(cfg)) > b
    ms = (ctypes.c_int32 * 3)(16, 32, 64)
    assert lib.mp_pan_workspace_bytes(1 << 14, ms, 3, ctypes.byref(cfg)) > 0
    bad = (ctypes.c_int32 * 1)(2)
    assert lib.mp_pan_workspace_bytes(1 << 14, bad, 1, ctypes.byref(cfg)) == 0
    assert lib.mp_batched_workspace_bytes(100000, 10, 128, ctypes.byref(cfg)) > 0
    assert lib.mp_backward_workspace_bytes(4096, 64) > 0
    cfg.prec = 7
    assert lib.mp_selfjoin_workspace_bytes(1 << 16, ctypes.byref(cfg)) == 0


def test_host_argument_checks_need_no_gpu(lib):
    """Every invalid call is rejected on the host before any CUDA call."""
    cfg = _lib.make_config(64)
    fake = 256 * 1024          # never dereferenced: the checks fail first
    E = _lib.MP_EINVAL
    assert lib.mp_selfjoin(None, 0, 4096, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    assert lib.mp_selfjoin(fake, 5, 4096, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    assert lib.mp_selfjoin(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake + 8, 1 << 30, None) == E
    cfg.m = 3
    assert lib.mp_selfjoin(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    cfg.m = 5000
    assert lib.mp_selfjoin(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    cfg.m = 64
    assert lib.mp_selfjoin(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake, 16, None) == _lib.MP_ENOMEM
    cfg.ez = -1.0
    assert lib.mp_selfjoin(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    cfg.ez = 0.5
    assert lib.mp_abjoin(fake, 4096, fake, 4096, 0, ctypes.byref(cfg), fake, fake, fake, None, fake,
                         1 << 30, None) == E
    ms = (ctypes.c_int32 * 2)(16, 3)
    assert lib.mp_pan(fake, 0, 4096, ms, 2, ctypes.byref(cfg), fake, fake, fake, 1 << 30, None) == E
    assert lib.mp_batched(fake, 0, 100, fake, fake, 0, 64, ctypes.byref(cfg), fake, fake, fake, fake,
                          1 << 30, None) == E
    assert lib.mp_backward(fake, 0, 4096, 2, fake, fake, fake, fake, 1 << 30, None) == E
    assert lib.mp_get_device_status(None, None) == E
    for code in range(7):
        assert lib.mp_status_string(code).decode()


def test_host_checks_of_the_newer_entry_points(lib):
    """Left/right, anytime, FLUSS and the non-normalised flag: invalid calls
    are rejected on the host, workspace queries answer without a GPU."""
    cfg = _lib.make_config(64)
    fake = 256 * 1024
    E = _lib.MP_EINVAL
    assert lib.mp_selfjoin_lr_workspace_bytes(4096, ctypes.byref(cfg)) > \
        lib.mp_selfjoin_workspace_bytes(4096, ctypes.byref(cfg))
    assert lib.mp_selfjoin_lr(fake, 0, 4096, ctypes.byref(cfg), fake, None, fake, fake, fake,
                              1 << 30, None) == E
    assert lib.mp_selfjoin_lr(fake, 0, 4096, ctypes.byref(cfg), fake, fake, fake, fake, fake + 8,
                              1 << 30, None) == E
    assert lib.mp_anytime_workspace_bytes(4096, ctypes.byref(cfg)) == \
        lib.mp_selfjoin_workspace_bytes(4096, ctypes.byref(cfg))
    assert lib.mp_anytime_begin(None, 0, 4096, ctypes.byref(cfg), 1, fake, 1 << 30, None) == E
    for f in (-0.1, 1.5, float("nan")):
        assert lib.mp_anytime_run(4096, ctypes.byref(cfg), f, fake, fake, fake, 1 << 30, None) == E
    assert lib.mp_fluss_workspace_bytes(0) == 0 and lib.mp_fluss_workspace_bytes(1 << 20) > 0
    assert lib.mp_fluss(None, 100, 0, 1, 0, fake, fake, fake, 1 << 20, None) == E
    assert lib.mp_fluss(fake, 100, -1, 1, 0, fake, fake, fake, 1 << 20, None) == E
    assert lib.mp_fluss(fake, 100, 0, 2, 0, fake, None, fake, 1 << 20, None) == E
    assert lib.mp_fluss(fake, 100, 0, 1, 0, fake, fake, fake, 16, None) == _lib.MP_ENOMEM
    raw1 = _lib.make_config(64, flags=_lib.MP_FLAG_RAW, variant=1)
    assert lib.mp_selfjoin_workspace_bytes(4096, ctypes.byref(raw1)) == 0   # default shape only
    raw0 = _lib.make_config(64, flags=_lib.MP_FLAG_RAW)
    assert lib.mp_selfjoin_workspace_bytes(4096, ctypes.byref(raw0)) > 0
