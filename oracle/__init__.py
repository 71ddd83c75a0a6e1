"""CPU FP64 brute-force oracle for the matrix-profile joins.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing in the library's
product path imports this package, and it imports nothing from the library.

The arithmetic lives in ``oracle.c`` (plain C, FP64, one pthread per host
core, built into ``liboracle.so`` next to it); this module only marshals
NumPy arrays through ctypes and composes whole-problem helpers (pan, batch)
out of the C self-join, each of which is the definition applied per problem.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False, cflags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile oracle.c into a shared library (gcc, FP64, no FMA contraction
    so x86 and Arm round the same way).  Returns the library path."""
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           *cflags, _SRC, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


def _bind(lib):
    lib.oracle_profile_length.restype = ctypes.c_int64
    lib.oracle_profile_length.argtypes = [ctypes.c_int64, ctypes.c_int32]
    lib.oracle_exclusion_zone.restype = ctypes.c_int64
    lib.oracle_exclusion_zone.argtypes = [ctypes.c_int32, ctypes.c_double]
    lib.oracle_window_stats.restype = ctypes.c_int
    lib.oracle_window_stats.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, _d, _d, _u8]
    lib.oracle_distance.restype = ctypes.c_double
    lib.oracle_distance.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_distance_ab.restype = ctypes.c_double
    lib.oracle_distance_ab.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_int64]
    lib.oracle_cov.restype = ctypes.c_double
    lib.oracle_cov.argtypes = [_d, _d, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_mpx_terms.restype = ctypes.c_int
    lib.oracle_mpx_terms.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, _d, _d]
    lib.oracle_selfjoin.restype = ctypes.c_int
    lib.oracle_selfjoin.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                    _i64, ctypes.c_int64, _d, _i64, _d, ctypes.c_int]
    lib.oracle_selfjoin_side.restype = ctypes.c_int
    lib.oracle_selfjoin_side.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int, _i64, ctypes.c_int64, _d,
                                         _i64, _d, ctypes.c_int]
    lib.oracle_arc_count_at.restype = ctypes.c_int64
    lib.oracle_arc_count_at.argtypes = [_i64, ctypes.c_int64, ctypes.c_int64]
    lib.oracle_arc_counts.restype = ctypes.c_int
    lib.oracle_arc_counts.argtypes = [_i64, ctypes.c_int64, _i64]
    lib.oracle_arc_counts_fast.restype = ctypes.c_int
    lib.oracle_arc_counts_fast.argtypes = [_i64, ctypes.c_int64, _i64]
    lib.oracle_cac.restype = ctypes.c_int
    lib.oracle_cac.argtypes = [_i64, ctypes.c_int64, ctypes.c_int64, _d]
    lib.oracle_segments.restype = ctypes.c_int
    lib.oracle_segments.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _i64]
    lib.oracle_selfjoin_diags.restype = ctypes.c_int
    lib.oracle_selfjoin_diags.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_int, _u8, _i64, ctypes.c_int64, _d, _i64, _d,
                                          ctypes.c_int]
    lib.oracle_join_raw.restype = ctypes.c_int
    lib.oracle_join_raw.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int, ctypes.c_int64, ctypes.c_int, _i64,
                                    ctypes.c_int64, _d, _i64, _d, ctypes.c_int]
    lib.oracle_abjoin.restype = ctypes.c_int
    lib.oracle_abjoin.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, ctypes.c_int32,
                                  _i64, ctypes.c_int64, _d, _i64, _d, ctypes.c_int]
    lib.oracle_grad.restype = ctypes.c_int
    lib.oracle_grad.argtypes = [_d, ctypes.c_int64, ctypes.c_int32, _i64, _d, _d]
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation tests swap in a deliberately broken build
            alt = os.environ.get("ORACLE_LIB")
            _lib = _bind(ctypes.CDLL(alt if alt else build()))
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a, t):
    return a.ctypes.data_as(t)


def profile_length(n: int, m: int, lib=None) -> int:
    return int((lib or load()).oracle_profile_length(n, m))


def exclusion_zone(m: int, ez: float = 0.5, lib=None) -> int:
    return int((lib or load()).oracle_exclusion_zone(m, ez))


def window_stats(x, m: int, lib=None):
    """(mu, sigma, flat) of every window, two-pass FP64."""
    lib = lib or load()
    x = _f64(x)
    l = profile_length(len(x), m, lib)
    mu, sig = np.empty(l), np.empty(l)
    flat = np.empty(l, dtype=np.uint8)
    lib.oracle_window_stats(_p(x, _d), len(x), m, _p(mu, _d), _p(sig, _d), _p(flat, _u8))
    return mu, sig, flat.astype(bool)


def distance(x, m: int, i: int, j: int, lib=None) -> float:
    x = _f64(x)
    return float((lib or load()).oracle_distance(_p(x, _d), len(x), m, i, j))


def distance_ab(a, b, m: int, i: int, j: int, lib=None) -> float:
    a, b = _f64(a), _f64(b)
    return float((lib or load()).oracle_distance_ab(_p(a, _d), len(a), _p(b, _d), len(b), m, i, j))


def cov(xa, xb, m: int, i: int, j: int, lib=None) -> float:
    xa, xb = _f64(xa), _f64(xb)
    return float((lib or load()).oracle_cov(_p(xa, _d), _p(xb, _d), m, i, j))


def mpx_terms(x, m: int, lib=None):
    """(df, dg) update terms of the diagonal recurrence, from their definition."""
    lib = lib or load()
    x = _f64(x)
    l = profile_length(len(x), m, lib)
    df, dg = np.empty(l), np.empty(l)
    rc = lib.oracle_mpx_terms(_p(x, _d), len(x), m, _p(df, _d), _p(dg, _d))
    if rc != 0:
        raise ValueError("oracle_mpx_terms failed")
    return df, dg


def selfjoin(x, m: int, ez: float = 0.5, rows=None, inclusive: bool = False,
             nthreads: int = 0, lib=None):
    """Brute-force self-join.  Returns (mp, pi, second) for `rows` (all rows
    when None); `second` is the second-smallest admissible distance."""
    lib = lib or load()
    x = _f64(x)
    l = profile_length(len(x), m, lib)
    rows = np.arange(l, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    excl = exclusion_zone(m, ez, lib)
    mp = np.empty(len(rows))
    pi = np.empty(len(rows), dtype=np.int64)
    sec = np.empty(len(rows))
    rc = lib.oracle_selfjoin(_p(x, _d), len(x), m, excl, int(inclusive), _p(rows, _i64), len(rows),
                             _p(mp, _d), _p(pi, _i64), _p(sec, _d), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_selfjoin failed ({rc})")
    return mp, pi, sec


def selfjoin_lr(x, m: int, ez: float = 0.5, rows=None, inclusive: bool = False,
                nthreads: int = 0, lib=None):
    """Brute-force left and right self-join profiles (candidates before / after
    each row).  Returns (mp_left, pi_left, sec_left, mp_right, pi_right, sec_right)."""
    lib = lib or load()
    x = _f64(x)
    l = profile_length(len(x), m, lib)
    rows = np.arange(l, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    excl = exclusion_zone(m, ez, lib)
    out = []
    for side in (-1, 1):
        mp = np.empty(len(rows))
        pi = np.empty(len(rows), dtype=np.int64)
        sec = np.empty(len(rows))
        rc = lib.oracle_selfjoin_side(_p(x, _d), len(x), m, excl, int(inclusive), side,
                                      _p(rows, _i64), len(rows), _p(mp, _d), _p(pi, _i64),
                                      _p(sec, _d), nthreads)
        if rc != 0:
            raise ValueError(f"oracle_selfjoin_side failed ({rc})")
        out += [mp, pi, sec]
    return tuple(out)


def arc_counts(pi, fast: bool = False, lib=None):
    """Arc count at every position: by the definition (O(l^2)) or by the
    difference-array form (O(l))."""
    lib = lib or load()
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    ac = np.empty(len(pi), dtype=np.int64)
    f = lib.oracle_arc_counts_fast if fast else lib.oracle_arc_counts
    if f(_p(pi, _i64), len(pi), _p(ac, _i64)) != 0:
        raise ValueError("oracle arc count failed")
    return ac


def arc_count_at(pi, k: int, lib=None) -> int:
    lib = lib or load()
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    return int(lib.oracle_arc_count_at(_p(pi, _i64), len(pi), int(k)))


def fluss(pi, m: int, num_segments: int = 2, edge=None, seg_excl=None, fast: bool = True,
          lib=None):
    """Corrected arc curve and segment boundaries (margins default to 5 m)."""
    lib = lib or load()
    l = len(pi)
    edge = 5 * m if edge is None else edge
    seg_excl = 5 * m if seg_excl is None else seg_excl
    ac = arc_counts(pi, fast=fast, lib=lib)
    cac = np.empty(l)
    if lib.oracle_cac(_p(ac, _i64), l, edge, _p(cac, _d)) != 0:
        raise ValueError("oracle_cac failed")
    seg = np.empty(num_segments, dtype=np.int64)
    if lib.oracle_segments(_p(cac, _d), l, num_segments, seg_excl, _p(seg, _i64)) != 0:
        raise ValueError("oracle_segments failed")
    return cac, seg


def selfjoin_diags(x, m: int, diag_ok, ez: float = 0.5, rows=None, inclusive: bool = False,
                   nthreads: int = 0, lib=None):
    """Brute-force self-join over the diagonals |i - j| with diag_ok set (an
    anytime run's best-so-far).  Returns (mp, pi, second)."""
    lib = lib or load()
    x = _f64(x)
    l = profile_length(len(x), m, lib)
    ok = np.ascontiguousarray(diag_ok, dtype=np.uint8)
    if len(ok) != l:
        raise ValueError("diag_ok needs l entries")
    rows = np.arange(l, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    excl = exclusion_zone(m, ez, lib)
    mp = np.empty(len(rows))
    pi = np.empty(len(rows), dtype=np.int64)
    sec = np.empty(len(rows))
    rc = lib.oracle_selfjoin_diags(_p(x, _d), len(x), m, excl, int(inclusive), _p(ok, _u8),
                                   _p(rows, _i64), len(rows), _p(mp, _d), _p(pi, _i64),
                                   _p(sec, _d), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_selfjoin_diags failed ({rc})")
    return mp, pi, sec


def join_raw(a, m: int, b=None, ez: float = 0.5, rows=None, inclusive: bool = False,
             nthreads: int = 0, lib=None):
    """Brute force with the non-normalised distance ||x_i - x_j||: a self-join
    of a (exclusion zone ez), or an AB-join of a against b.  Returns (mp, pi, second)."""
    lib = lib or load()
    a = _f64(a)
    bb = a if b is None else _f64(b)
    la = profile_length(len(a), m, lib)
    rows = np.arange(la, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    excl = exclusion_zone(m, ez, lib)
    mp = np.empty(len(rows))
    pi = np.empty(len(rows), dtype=np.int64)
    sec = np.empty(len(rows))
    rc = lib.oracle_join_raw(_p(a, _d), len(a), _p(bb, _d), len(bb), m, int(b is not None), excl,
                             int(inclusive), _p(rows, _i64), len(rows), _p(mp, _d), _p(pi, _i64),
                             _p(sec, _d), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_join_raw failed ({rc})")
    return mp, pi, sec


def abjoin(a, b, m: int, rows=None, nthreads: int = 0, lib=None):
    """Brute-force AB-join: for windows `rows` of a, the nearest window of b."""
    lib = lib or load()
    a, b = _f64(a), _f64(b)
    la = profile_length(len(a), m, lib)
    rows = np.arange(la, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    mp = np.empty(len(rows))
    pi = np.empty(len(rows), dtype=np.int64)
    sec = np.empty(len(rows))
    rc = lib.oracle_abjoin(_p(a, _d), len(a), _p(b, _d), len(b), m, _p(rows, _i64), len(rows),
                           _p(mp, _d), _p(pi, _i64), _p(sec, _d), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_abjoin failed ({rc})")
    return mp, pi, sec


def grad(x, m: int, pi, g, lib=None) -> np.ndarray:
    """dL/dx for L = sum_i g_i MP_i with the argmin pairs (i, pi[i]) held fixed."""
    lib = lib or load()
    x = _f64(x)
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    g = _f64(g)
    out = np.empty(len(x))
    rc = lib.oracle_grad(_p(x, _d), len(x), m, _p(pi, _i64), _p(g, _d), _p(out, _d))
    if rc != 0:
        raise ValueError("oracle_grad failed")
    return out


def pan(x, ms, ez: float = 0.5, rows_per_m=None, nthreads: int = 0, lib=None):
    """Pan matrix profile: the self-join at every window size in `ms`.
    Returns a list of (rows, mp, pi, second) per window size."""
    out = []
    for k, m in enumerate(ms):
        rows = None if rows_per_m is None else rows_per_m[k]
        l = profile_length(len(x), int(m), lib)
        r = np.arange(l, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
        mp, pi, sec = selfjoin(x, int(m), ez, r, nthreads=nthreads, lib=lib)
        out.append((r, mp, pi, sec))
    return out


def batched(values, offsets, ms, ez: float = 0.5, series=None, rows_per_series=None,
            nthreads: int = 0, lib=None):
    """Self-join of each series values[offsets[b]:offsets[b+1]] with window
    ms[b].  Returns {b: (rows, mp, pi, second)} for the requested series."""
    series = range(len(ms)) if series is None else series
    out = {}
    for k, b in enumerate(series):
        xb = values[offsets[b]:offsets[b + 1]]
        rows = None if rows_per_series is None else rows_per_series[k]
        l = profile_length(len(xb), int(ms[b]), lib)
        r = np.arange(l, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
        mp, pi, sec = selfjoin(xb, int(ms[b]), ez, r, nthreads=nthreads, lib=lib)
        out[b] = (r, mp, pi, sec)
    return out
