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
