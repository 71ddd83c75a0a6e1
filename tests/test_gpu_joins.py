"""GPU parity of the AB-join, the batched ragged joins, the pan profile and
the backward pass (CUDA path through the C ABI vs the CPU oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_12626_gb300 import synth

from _parity import check_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-3}


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12626_gb300 import api, build
    build.build()
    api.init()
    return api


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_abjoin_small_with_flats_both_sides(mp, prec):
    a = synth.random_walk(2500, seed=11)
    b, flats = synth.mixed_with_flats(1800, 24, seed=12, block=256, n_flat=3)
    b = b.astype(np.float64)
    m = 24
    ma, pa, mb, pb = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec=prec, tile_rows=512,
                                                           check_status=True))
    mo, po, so = oracle.abjoin(a, b, m)
    check_rows(a, m, np.arange(len(mo)), ma, pa, mo, po, so, TOL[prec], y=b)
    mo, po, so = oracle.abjoin(b, a, m)
    check_rows(b, m, np.arange(len(mo)), mb, pb, mo, po, so, TOL[prec], y=a)
    s = int(flats[0]) + 5                                  # a flat window of b
    assert mb[s] == math.sqrt(2 * m) and pb[s] == 0


def test_abjoin_symmetry_and_one_sided(mp):
    a = synth.random_walk(3000, seed=13)
    b = synth.random_walk(2000, seed=14)
    m = 50
    ma, pa, mb, pb = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec="fp64"))
    ma2, pa2, mb2, pb2 = (t.cpu().numpy() for t in mp.abjoin(_t(b), _t(a), m, prec="fp64"))
    np.testing.assert_allclose(mb, ma2, atol=1e-9)
    np.testing.assert_allclose(ma, mb2, atol=1e-9)
    assert (pb == pa2).mean() > 0.999 and (pa == pb2).mean() > 0.999
    ma3, pa3, mb3, pb3 = mp.abjoin(_t(a), _t(b), m, prec="fp64", both=False)
    assert mb3 is None and pb3 is None
    np.testing.assert_allclose(ma3.cpu().numpy(), ma, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_ragged_all_rows(mp, prec):
    values, offsets, ms = synth.ragged_batch(40, seed=15, len_lo=60, len_hi=3000)
    g_mp, g_pi, oo = mp.batched(_t(values), _t(offsets), _t(ms), prec=prec, tile_rows=512,
                                check_status=True)
    g_mp, g_pi = g_mp.cpu().numpy(), g_pi.cpu().numpy()
    ref = oracle.batched(values.astype(np.float64), offsets, ms)
    for b, (rows, mo, po, so) in ref.items():
        o = int(offsets[b])
        xb = values[offsets[b]:offsets[b + 1]].astype(np.float64)
        E = oracle.exclusion_zone(int(ms[b]))
        check_rows(xb, int(ms[b]), rows, g_mp[o:o + len(rows)], g_pi[o:o + len(rows)], mo, po, so,
                   TOL[prec], excl=E)


def test_batched_degenerate_series(mp):
    """Series shorter than their window, and series with l <= E."""
    lens = [100, 10, 40, 3000, 33]
    ms_ = np.array([32, 16, 32, 64, 32], np.int32)
    rng = np.random.default_rng(16)
    values = np.concatenate([np.cumsum(rng.standard_normal(k)) for k in lens])
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    g_mp, g_pi, _ = mp.batched(_t(values), _t(offsets), _t(ms_), prec="fp64", check_status=False)
    g_mp, g_pi = g_mp.cpu().numpy(), g_pi.cpu().numpy()
    for b, k in enumerate(lens):
        l = k - int(ms_[b]) + 1
        if l <= 0:
            continue
        xb = values[offsets[b]:offsets[b + 1]]
        mo, po, so = oracle.selfjoin(xb, int(ms_[b]))
        o = int(offsets[b])
        check_rows(xb, int(ms_[b]), np.arange(l), g_mp[o:o + l], g_pi[o:o + l], mo, po, so, 1e-9,
                   excl=oracle.exclusion_zone(int(ms_[b])))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pan_small_all_rows(mp, prec):
    x = synth.random_walk(2000, seed=17)
    ms = [8, 13, 16, 40, 77, 128]
    pan, pi = mp.pan(_t(x), ms, prec=prec, tile_rows=512, check_status=True)
    pan, pi = pan.cpu().numpy(), pi.cpu().numpy()
    assert pan.shape == (len(ms), 2000 - 8 + 1)
    for k, m in enumerate(ms):
        l = 2000 - m + 1
        mo, po, so = oracle.selfjoin(x, m)
        check_rows(x, m, np.arange(l), pan[k, :l], pi[k, :l], mo, po, so, TOL[prec],
                   excl=oracle.exclusion_zone(m))
        assert np.isinf(pan[k, l:]).all() and (pi[k, l:] == -1).all()
    pan_n, _ = mp.pan(_t(x), ms, prec="fp64", normalize=True)
    pan_n = pan_n.cpu().numpy()
    for k, m in enumerate(ms):
        l = 2000 - m + 1
        mo, _, _ = oracle.selfjoin(x, m)
        np.testing.assert_allclose(pan_n[k, :l], mo / math.sqrt(2 * m), atol=1e-9)


def test_backward_matches_oracle_gradient(mp):
    n, m = 2048, 32
    x = synth.random_walk(n, seed=18)
    mp_g, pi_g = mp.selfjoin(_t(x), m, prec="fp64")
    pi_np = pi_g.cpu().numpy()
    g = np.ones(n - m + 1)
    g[np.argsort(-mp_g.cpu().numpy(), kind="stable")[:16]] += 1.0 / 16
    gx = mp.backward(_t(x), m, pi_g, _t(g)).cpu().numpy()
    ref = oracle.grad(x, m, pi_np, g)
    err = np.linalg.norm(gx - ref) / np.linalg.norm(ref)
    assert err <= 1e-9, err


def test_autograd_function(mp):
    n, m = 4096, 64
    x = torch.tensor(synth.random_walk(n, seed=19), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    prof, pi = mp.matrix_profile(x, m, 0.5, "fp64")
    loss = prof.sum() + prof.topk(16).values.mean()
    loss.backward()
    g = np.ones(n - m + 1)
    g[torch.topk(prof.detach(), 16).indices.cpu().numpy()] += 1.0 / 16
    ref = oracle.grad(x.detach().cpu().numpy(), m, pi.cpu().numpy(), g)
    err = np.linalg.norm(x.grad.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-9, err
