"""Write the stored oracle answers of the full-size parity tests.

The full-size workloads are too large for the CPU oracle to finish inside a
GPU test run (the B side of the AB-join alone is 4,096 rows, each against
2^21 windows of 512 samples), so their sampled rows are computed here, once,
by the oracle alone, and stored with a fingerprint of the input they were
computed from.  A test regenerates the same seeded input, and uses the stored
answers only when the fingerprint matches; otherwise it runs the oracle
itself.  Nothing here touches the CUDA path.

    python tests/golden/make_oracle_samples.py [c2] [c3]

Files (NumPy .npz, next to this script):
  c2_planted_n2p20_m256.npz   self-join of the planted 2^20 walk (seed 2024),
                              m = 256: 4,096 seeded rows plus every planted
                              row +-4 and the discord's rows +-4
  c3_ab_n2p21_n2p19_m512.npz  AB-join of a 2^21 walk (seed 51) against the
                              2^19 walk / white-noise mix with ten flat
                              stretches (seed 52), m = 512: 4,096 rows of A,
                              4,096 rows of B plus every row within 4 of a
                              flat stretch's transitions
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from _golden import c2_inputs, c2_rows, c3_inputs, c3_rows, fingerprint  # noqa: E402

C2_FILE = os.path.join(HERE, "c2_planted_n2p20_m256.npz")
C3_FILE = os.path.join(HERE, "c3_ab_n2p21_n2p19_m512.npz")


def make_c2() -> None:
    x, info, m = c2_inputs()
    rows = c2_rows(x, info, m)
    x64 = x.astype(np.float64)
    t0 = time.time()
    mp, pi, sec = oracle.selfjoin(x64, m, rows=rows)
    print(f"c2: {len(rows)} rows in {time.time() - t0:.0f} s")
    np.savez_compressed(C2_FILE, fingerprint=fingerprint(x), rows=rows, mp=mp, pi=pi, sec=sec)


def make_c3() -> None:
    a, b, flats, m = c3_inputs()
    rows_a, rows_b = c3_rows(a, b, flats, m)
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    t0 = time.time()
    mp_a, pi_a, sec_a = oracle.abjoin(a64, b64, m, rows=rows_a)
    print(f"c3 A: {len(rows_a)} rows in {time.time() - t0:.0f} s")
    t0 = time.time()
    mp_b, pi_b, sec_b = oracle.abjoin(b64, a64, m, rows=rows_b)
    print(f"c3 B: {len(rows_b)} rows in {time.time() - t0:.0f} s")
    np.savez_compressed(C3_FILE, fingerprint=fingerprint(a, b), rows_a=rows_a, mp_a=mp_a,
                        pi_a=pi_a, sec_a=sec_a, rows_b=rows_b, mp_b=mp_b, pi_b=pi_b, sec_b=sec_b)


if __name__ == "__main__":
    oracle.build()
    which = sys.argv[1:] or ["c2", "c3"]
    if "c2" in which:
        make_c2()
    if "c3" in which:
        make_c3()
