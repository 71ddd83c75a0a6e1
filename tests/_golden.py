"""Full-size workloads of the parity tests, their sampled rows, and the
oracle's answers for them.

The answers come from the CPU oracle only: either computed here, or read
from a file that ``tests/golden/make_oracle_samples.py`` wrote by running the
oracle on the same seeded input.  A stored file is used only when the
fingerprint of the input it was computed from matches the input regenerated
here (same seed, same generator); otherwise the oracle runs now.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

import oracle
from paper_1904_12626_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fingerprint(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode() + str(a.shape).encode() + a.tobytes())
    return h.hexdigest()


# ---- planted self-join: 2^20 float32 walk, 3 motif pairs, 1 discord, m = 256

def c2_inputs():
    m = 256
    x, info = synth.planted_walk(1 << 20, m, seed=2024)
    return x, info, m


def c2_planted_rows(info):
    rows = []
    for p1, p2 in info["pairs"]:
        for p in (p1, p2):
            rows += range(p - 4, p + 5)
    d = info["discord"]
    rows += range(d - 4, d + 5)
    return np.asarray(rows, dtype=np.int64)


def c2_rows(x, info, m):
    """4,096 seeded rows plus every planted row +-4."""
    l = len(x) - m + 1
    return np.unique(np.concatenate([synth.sample_rows(l, 4096, seed=7), c2_planted_rows(info)]))


# ---- AB-join: 2^21 walk against a 2^19 walk / white-noise mix with flats, m = 512

def c3_inputs():
    m = 512
    a = synth.random_walk(1 << 21, seed=51, dtype=np.float32)
    b, flats = synth.mixed_with_flats(1 << 19, m, seed=52)
    return a, b, flats, m


def c3_flat_rows(flats, m, lb, flat_len=None):
    """Rows of B within 4 of each flat stretch's transitions: the first window
    that reaches the stretch, the first and last fully flat window, and the
    first window past it."""
    F = 2 * m if flat_len is None else flat_len
    rows = []
    for s in flats:
        s = int(s)
        for t in (s - m + 1, s, s + F - m, s + F):
            rows += [r for r in range(t - 4, t + 5) if 0 <= r < lb]
    return np.asarray(rows, dtype=np.int64)


def c3_rows(a, b, flats, m):
    la, lb = len(a) - m + 1, len(b) - m + 1
    rows_a = synth.sample_rows(la, 4096, seed=53)
    rows_b = np.unique(np.concatenate([synth.sample_rows(lb, 4096, seed=54),
                                       c3_flat_rows(flats, m, lb)]))
    return rows_a, rows_b


# ---- loading with a fallback to the oracle itself

def _load(name: str, fp: str):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        return None
    z = np.load(path)
    if str(z["fingerprint"]) != fp:
        return None
    return {k: z[k] for k in z.files}


def c2_oracle(x, info, m):
    """(rows, mp, pi, sec) of the oracle on c2_rows, and whether they came
    from the stored file."""
    rows = c2_rows(x, info, m)
    z = _load("c2_planted_n2p20_m256.npz", fingerprint(x))
    if z is not None and np.array_equal(z["rows"], rows):
        return (rows, z["mp"], z["pi"], z["sec"]), True
    mp, pi, sec = oracle.selfjoin(x.astype(np.float64), m, rows=rows)
    return (rows, mp, pi, sec), False


def c3_oracle(a, b, flats, m):
    """((rows_a, mp, pi, sec), (rows_b, mp, pi, sec)) and whether stored."""
    rows_a, rows_b = c3_rows(a, b, flats, m)
    z = _load("c3_ab_n2p21_n2p19_m512.npz", fingerprint(a, b))
    if z is not None and np.array_equal(z["rows_a"], rows_a) and np.array_equal(z["rows_b"], rows_b):
        return ((rows_a, z["mp_a"], z["pi_a"], z["sec_a"]),
                (rows_b, z["mp_b"], z["pi_b"], z["sec_b"])), True
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    ra = (rows_a, *oracle.abjoin(a64, b64, m, rows=rows_a))
    rb = (rows_b, *oracle.abjoin(b64, a64, m, rows=rows_b))
    return (ra, rb), False
