"""Host-side pieces of the benchmark (no GPU): the oracle sample it times
also measures the GPU profile's error, so that sample and the error
summary must be consistent."""
import numpy as np

import bench
import oracle
from paper_1904_12626_gb300 import synth


def test_cpu_oracle_sample_and_accuracy():
    x = synth.random_walk(3000, seed=5)
    m, E = 32, 16
    rate, rows, secs, cores, res = bench.cpu_oracle_rate(x, m, E, target_s=0.05)
    r, mo, po, so = res
    assert rate > 0 and cores >= 1 and len(r) == rows == len(mo) == len(po) == len(so)
    full_mp, full_pi, _ = oracle.selfjoin(x, m)
    acc = bench.accuracy(res, full_mp, full_pi)
    assert acc["max_abs_dmp"] == 0.0 and acc["pi_equal_on_separated"] and acc["finite_pattern_equal"]
    assert 0 < acc["separated_rows"] <= rows
    # a profile off by 2e-4 on one sampled row, and a wrong index on a separated row
    mp2, pi2 = full_mp.copy(), full_pi.copy()
    mp2[r[0]] += 2e-4
    sep = np.nonzero((so - mo) > 1e-3)[0]
    pi2[r[sep[0]]] = (pi2[r[sep[0]]] + 1000) % len(pi2)
    acc = bench.accuracy(res, mp2, pi2)
    assert abs(acc["max_abs_dmp"] - 2e-4) < 1e-12 and not acc["pi_equal_on_separated"]


def test_workspace_header_fields():
    """The bench reads the plan's tile count (bytes 24..31) and band width
    (bytes 20..23) from the workspace header; the offsets follow the header's
    layout: status, pad, ticket (8 bytes), bands (4), band width (4), tiles (8)."""
    import torch
    ws = torch.zeros(256, dtype=torch.uint8)
    ws[20:24] = torch.from_numpy(np.array([1024], dtype=np.int32).view(np.uint8))
    ws[24:32] = torch.from_numpy(np.array([48520], dtype=np.uint64).view(np.uint8))
    ws[16:20] = torch.from_numpy(np.array([777], dtype=np.int32).view(np.uint8))
    assert bench.workspace_tile_diags(ws) == 1024
    assert bench.workspace_tiles(ws) == 48520
