"""GPU parity of mp_stats (compensated FP64 window statistics) against the oracle."""
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


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("offset", [0.0, 1.0e6])
def test_stats_match_definitions(mp, dtype, offset):
    m = 96
    x = synth.random_walk(20000, seed=41).astype(np.float64) + offset
    x[5000:5200] = x[4999]                      # flat windows
    x = x.astype(dtype)
    x64 = x.astype(np.float64)
    mu, invn, df, dg, flat = (t.cpu().numpy() for t in mp.stats(torch.from_numpy(x).cuda(), m))
    mu_o, sig_o, flat_o = oracle.window_stats(x64, m)
    df_o, dg_o = oracle.mpx_terms(x64, m)
    np.testing.assert_array_equal(flat.astype(bool), flat_o)
    scale = np.abs(x64).max() + 1.0
    np.testing.assert_allclose(mu, mu_o, rtol=0, atol=1e-15 * scale * 4)
    nf = ~flat_o
    inv_o = 1.0 / (sig_o[nf] * math.sqrt(m))
    np.testing.assert_allclose(invn[nf], inv_o, rtol=1e-12 if offset == 0 else 1e-9)
    assert np.all(invn[flat_o] == 0.0)
    np.testing.assert_allclose(df, df_o, rtol=0, atol=1e-15 * scale * 4)
    np.testing.assert_allclose(dg, dg_o, rtol=0, atol=1e-13 * scale)


def test_stats_recurrence_identity_exact(mp):
    """On small integers with a power-of-two window every term is exact, so
    the GPU's df/dg must reproduce the oracle's direct covariances exactly."""
    rng = np.random.default_rng(42)
    x = rng.integers(-30, 31, size=3000).astype(np.float64)
    m = 64
    mu, invn, df, dg, flat = (t.cpu().numpy() for t in mp.stats(torch.from_numpy(x).cuda(), m))
    for _ in range(300):
        i, j = (int(v) for v in rng.integers(1, len(x) - m + 1, 2))
        lhs = oracle.cov(x, x, m, i, j) - oracle.cov(x, x, m, i - 1, j - 1)
        assert lhs == df[i] * dg[j] + df[j] * dg[i]
