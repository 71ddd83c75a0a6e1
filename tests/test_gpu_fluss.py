"""GPU parity of semantic segmentation (FLUSS, Sec. 3.4.2) through the C ABI
against the oracle: the arc counts are integers, so the corrected arc curve
(the same double expression on both sides) and the boundaries must match
exactly."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    return api


def _regimes(seed=31):
    rng = np.random.default_rng(seed)
    t = np.arange(3000)
    a = np.sin(2 * math.pi * t / 40.0)
    b = ((t % 25) / 25.0) * 2.0 - 1.0
    return np.concatenate([a, b]) + 0.05 * rng.standard_normal(6000)


def test_fluss_on_oracle_profile_index(mp):
    x = _regimes()
    m = 40
    _, pi, _ = oracle.selfjoin(x, m)
    cac_o, seg_o = oracle.fluss(pi, m, num_segments=3, fast=False)
    cac, seg = mp.fluss(torch.from_numpy(pi).cuda(), m, num_segments=3, check_status=True)
    np.testing.assert_array_equal(cac.cpu().numpy(), cac_o)
    np.testing.assert_array_equal(seg.cpu().numpy(), seg_o)
    assert abs(int(seg_o[0]) - 3000) <= 2 * m


@pytest.mark.parametrize("seed", [1, 2])
def test_fluss_random_index_full_size(mp, seed):
    """l = 2^20 seeded random neighbours with gaps and self arcs (several scan
    tiles, a ragged tail): every position against the O(l) oracle form, and
    sampled positions against the definition itself."""
    rng = np.random.default_rng(seed)
    l = (1 << 20) - 255
    pi = rng.integers(0, l, size=l)
    pi[rng.random(l) < 0.05] = -1
    pi[::1000] = np.arange(0, l, 1000)                 # self arcs: no crossing
    m = 256
    cac, seg = mp.fluss(torch.from_numpy(pi).cuda(), m, num_segments=4, check_status=True)
    cac, seg = cac.cpu().numpy(), seg.cpu().numpy()
    cac_o, seg_o = oracle.fluss(pi, m, num_segments=4, fast=True)
    np.testing.assert_array_equal(cac, cac_o)
    np.testing.assert_array_equal(seg, seg_o)
    ks = synth.sample_rows(l, 6, seed=seed + 10)
    for k in ks:
        ac = oracle.arc_count_at(pi, int(k))
        iac = 2.0 * k * (l - k) / l
        want = 1.0 if (k < 5 * m or k >= l - 5 * m or iac == 0) else min(ac / iac, 1.0)
        assert cac[k] == want


def test_fluss_edge_cases(mp):
    from paper_1904_12626_gb300 import _lib
    # one window, no neighbour
    cac, seg = mp.fluss(torch.tensor([-1], dtype=torch.int64, device="cuda"), 4, num_segments=2)
    assert cac.cpu().tolist() == [1.0] and seg.cpu().tolist() == [0, -1]
    # margins wider than the curve: all ones; more segments than positions
    pi = torch.tensor([3, 2, 1, 0, 2], dtype=torch.int64, device="cuda")
    cac, seg = mp.fluss(pi, 4, num_segments=7, edge=3, seg_excl=1)
    assert cac.cpu().tolist() == [1.0] * 5
    assert seg.cpu().tolist() == [0, 1, 2, 3, 4, -1, -1]
    # an index outside the profile is reported through the workspace status
    bad = torch.tensor([1, 0, 9], dtype=torch.int64, device="cuda")
    with pytest.raises(_lib.MPError) as e:
        mp.fluss(bad, 4, num_segments=1, check_status=True)
    assert e.value.code == _lib.MP_EINVAL


def test_fluss_end_to_end_fp32(mp):
    """GPU self-join (FP32-mixed) then GPU segmentation finds the change."""
    x = _regimes(seed=32).astype(np.float32)
    m = 40
    _, pi = mp.selfjoin(torch.from_numpy(x).cuda(), m, prec="fp32")
    cac, seg = mp.fluss(pi, m, num_segments=1)
    assert abs(int(seg.cpu()[0]) - 3000) <= 2 * m
