"""ctypes binding of libmpgb.so (the C ABI declared in include/mp.h).

Argument marshalling only: every step of every join runs in the library's
CUDA kernels.  The shared library is built in-tree by ``build.py``; if it is
missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmpgb.so")

MP_OK, MP_EINVAL, MP_EINVAL_DATA, MP_ENOMEM, MP_ECUDA, MP_ETIMEOUT, MP_EUNSUPPORTED, MP_EBOUNDS = range(8)
MP_F32, MP_F64 = 0, 1
MP_PREC_FP64, MP_PREC_FP32_MIXED = 0, 1
MP_FLAG_EXCL_INCLUSIVE = 0x1
MP_FLAG_NO_REFINE = 0x2
MP_FLAG_PAN_NORMALIZE = 0x4
MP_FLAG_RAW = 0x8


class MPConfig(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("ez", ctypes.c_double), ("prec", ctypes.c_int32),
                ("anchor_every", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class MPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_cfgp = ctypes.POINTER(MPConfig)
_i32p = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes)
SIGNATURES = {
    "mp_config_default": (None, [_cfgp, _i32]),
    "mp_profile_length": (_i64, [_i64, _i32]),
    "mp_exclusion_zone": (_i64, [_i32, _dbl]),
    "mp_version": (ctypes.c_char_p, []),
    "mp_variant_count": (_i32, [_i32]),
    "mp_variant_info": (ctypes.c_int, [_i32, _i32, _i32p, _i32p]),
    "mp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mp_init": (ctypes.c_int, [_i32]),
    "mp_stats": (ctypes.c_int, [_vp, _i32, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mp_selfjoin_workspace_bytes": (_sz, [_i64, _cfgp]),
    "mp_selfjoin": (ctypes.c_int, [_vp, _i32, _i64, _cfgp, _vp, _vp, _vp, _sz, _vp]),
    "mp_selfjoin_lr_workspace_bytes": (_sz, [_i64, _cfgp]),
    "mp_fluss_workspace_bytes": (_sz, [_i64]),
    "mp_anytime_workspace_bytes": (_sz, [_i64, _cfgp]),
    "mp_anytime_begin": (ctypes.c_int, [_vp, _i32, _i64, _cfgp, ctypes.c_uint64, _vp, _sz, _vp]),
    "mp_anytime_run": (ctypes.c_int, [_i64, _cfgp, _dbl, _vp, _vp, _vp, _sz, _vp]),
    "mp_fluss": (ctypes.c_int, [_vp, _i64, _i64, _i32, _i64, _vp, _vp, _vp, _sz, _vp]),
    "mp_selfjoin_lr": (ctypes.c_int, [_vp, _i32, _i64, _cfgp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "mp_selfjoin_noalloc": (ctypes.c_int, [_vp, _i32, _i64, _cfgp, _vp, _vp, _vp]),
    "mp_selfjoin_noalloc_max_n": (_i64, [_cfgp]),
    "mp_selfjoin_noalloc_device_status": (ctypes.c_int, [_vp]),
    "mp_abjoin_workspace_bytes": (_sz, [_i64, _i64, _cfgp]),
    "mp_abjoin": (ctypes.c_int, [_vp, _i64, _vp, _i64, _i32, _cfgp, _vp, _vp, _vp, _vp, _vp, _sz,
                                 _vp]),
    "mp_batched_workspace_bytes": (_sz, [_i64, _i32, _i32, _cfgp]),
    "mp_batched": (ctypes.c_int, [_vp, _i32, _i64, _vp, _vp, _i32, _i32, _cfgp, _vp, _vp, _vp, _vp,
                                  _sz, _vp]),
    "mp_pan_workspace_bytes": (_sz, [_i64, _i32p, _i32, _cfgp]),
    "mp_pan": (ctypes.c_int, [_vp, _i32, _i64, _i32p, _i32, _cfgp, _vp, _vp, _vp, _sz, _vp]),
    "mp_backward_workspace_bytes": (_sz, [_i64, _i32]),
    "mp_backward": (ctypes.c_int, [_vp, _i32, _i64, _i32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "mp_timing_enable": (ctypes.c_int, [_i32]),
    "mp_timing_last_ms": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float)]),
    "mp_probe_fp64_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "mp_get_device_status": (ctypes.c_int, [_vp, _vp]),
}


def load(path: str | None = None):
    """Load libmpgb.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1904_12626_gb300.build.build() "
                               "(the CUDA library is the only compute path)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load().mp_status_string(code).decode()
    except Exception:  # noqa: BLE001 - message only
        return f"status {code}"


def check(code: int, where: str) -> None:
    if code != MP_OK:
        raise MPError(code, where)


def make_config(m: int, ez: float = 0.5, prec: str = "fp32", anchor_every: int = 0,
                tile_rows: int = 0, variant: int = -1, flags: int = 0) -> MPConfig:
    cfg = MPConfig()
    load().mp_config_default(ctypes.byref(cfg), int(m))
    cfg.ez = float(ez)
    if prec in ("fp32", "fp32_mixed", MP_PREC_FP32_MIXED):
        cfg.prec = MP_PREC_FP32_MIXED
    elif prec in ("fp64", MP_PREC_FP64):
        cfg.prec = MP_PREC_FP64
    else:
        raise ValueError(f"unknown precision {prec!r}")
    cfg.anchor_every = int(anchor_every)
    cfg.tile_rows = int(tile_rows)
    cfg.variant = int(variant)
    cfg.flags = int(flags)
    return cfg
