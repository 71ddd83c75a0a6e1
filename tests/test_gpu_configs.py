"""GPU parity at the full workload sizes (sampled rows, checked one by one
against the oracle), in the launch configurations the library uses by
default:

* AB-join of a 2^21 random walk against a 2^19 white-noise / random-walk
  mix with ten flat stretches of 2m, m = 512, both directions, plus the
  join symmetry A-B vs B-A;
* 4096 ragged random walks (lengths 1000..65536, m in {32, 64, 128}) in one
  batched launch;
* the pan profile of a 2^16 random walk over 64 geometric window sizes
  16..1024;
* the gradient of sum(MP) + mean(top-16 MP) on a 2^16 series, m = 128.
"""
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


@pytest.fixture(scope="module")
def ab_inputs():
    m = 512
    a = synth.random_walk(1 << 21, seed=51, dtype=np.float32)
    b, flats = synth.mixed_with_flats(1 << 19, m, seed=52)
    return a, b, flats, m


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_abjoin_full_size_sampled(mp, ab_inputs, prec):
    a, b, flats, m = ab_inputs
    ma, pa, mb, pb = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec=prec,
                                                           check_status=True))
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    la, lb = len(a) - m + 1, len(b) - m + 1
    rows_a = synth.sample_rows(la, 96, seed=53)
    near_flat = []
    for s in flats:                                # windows touching each flat stretch's edges
        for r in (s - m, s - m + 1, s - 1, s, s + 1, s + 2 * m - m, s + 2 * m - m + 1, s + 2 * m):
            if 0 <= r < lb:
                near_flat.append(r)
    rows_b = np.unique(np.concatenate([synth.sample_rows(lb, 96, seed=54), near_flat]))
    mo, po, so = oracle.abjoin(a64, b64, m, rows=rows_a)
    check_rows(a64, m, rows_a, ma, pa, mo, po, so, TOL[prec], y=b64)
    mo, po, so = oracle.abjoin(b64, a64, m, rows=rows_b)
    check_rows(b64, m, rows_b, mb, pb, mo, po, so, TOL[prec], y=a64)
    for s in flats:                                # fully flat windows: closed form
        assert mb[s + 1] == math.sqrt(2 * m) and pb[s + 1] == 0


def test_abjoin_symmetry_full_size(mp, ab_inputs):
    a, b, _, m = ab_inputs
    ma, pa, mb, pb = mp.abjoin(_t(a), _t(b), m, prec="fp32")
    ma2, pa2, mb2, pb2 = mp.abjoin(_t(b), _t(a), m, prec="fp32")
    assert float((mb - ma2).abs().max()) <= 1e-9       # both refined in FP64 from the same pairs
    assert float((ma - mb2).abs().max()) <= 1e-9
    assert float((pb == pa2).double().mean()) > 0.9999
    assert float((pa == pb2).double().mean()) > 0.9999


@pytest.mark.parametrize("prec", ["fp32"])
def test_batched_4096_ragged_sampled(mp, prec):
    values, offsets, ms = synth.ragged_batch(4096, seed=55)
    g_mp, g_pi, _ = mp.batched(_t(values), _t(offsets), _t(ms), prec=prec, check_status=True)
    g_mp, g_pi = g_mp.cpu().numpy(), g_pi.cpu().numpy()
    rng = np.random.default_rng(56)
    series = np.sort(rng.choice(len(ms), 48, replace=False))
    for b in series:
        n_b = int(offsets[b + 1] - offsets[b])
        m = int(ms[b])
        l = n_b - m + 1
        rows = synth.sample_rows(l, 128, seed=int(b))
        xb = values[offsets[b]:offsets[b + 1]].astype(np.float64)
        mo, po, so = oracle.selfjoin(xb, m, rows=rows)
        o = int(offsets[b])
        check_rows(xb, m, rows, g_mp[o:o + l], g_pi[o:o + l], mo, po, so, TOL[prec],
                   excl=oracle.exclusion_zone(m))


@pytest.mark.parametrize("prec", ["fp32"])
def test_pan_64_sizes_sampled(mp, prec):
    n = 1 << 16
    x = synth.random_walk(n, seed=57, dtype=np.float32)
    ms = synth.pan_windows()
    assert len(set(ms.tolist())) == 64 and ms[0] == 16 and ms[-1] == 1024
    pan, pi = mp.pan(_t(x), ms, prec=prec, check_status=True)
    pan, pi = pan.cpu().numpy(), pi.cpu().numpy()
    x64 = x.astype(np.float64)
    for k in range(0, 64, 3):
        m = int(ms[k])
        l = n - m + 1
        rows = synth.sample_rows(l, 24, seed=k)
        mo, po, so = oracle.selfjoin(x64, m, rows=rows)
        check_rows(x64, m, rows, pan[k, :l], pi[k, :l], mo, po, so, TOL[prec],
                   excl=oracle.exclusion_zone(m))
        assert np.isinf(pan[k, l:]).all() and (pi[k, l:] == -1).all()


def test_gradient_2p16(mp):
    """loss = sum(MP) + mean of the top-16 MP values; the GPU gradient through
    the argmin pairs against the oracle's closed form at the same pairs."""
    n, m = 1 << 16, 128
    x = torch.tensor(synth.random_walk(n, seed=58, dtype=np.float32), device="cuda",
                     requires_grad=True)
    prof, pi = mp.matrix_profile(x, m, 0.5, "fp32")
    loss = prof.sum() + prof.topk(16).values.mean()
    loss.backward()
    g = np.ones(n - m + 1)
    g[torch.topk(prof.detach(), 16).indices.cpu().numpy()] += 1.0 / 16
    ref = oracle.grad(x.detach().cpu().numpy().astype(np.float64), m, pi.cpu().numpy(), g)
    gx = x.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(gx - ref) / np.linalg.norm(ref)
    assert err <= 1e-3, err


def test_gradient_central_differences_2048(mp):
    """FP64 central differences (h = 1e-6) of the oracle's MP on the first
    2048 samples run as their own series, against the GPU gradient; a seeded
    sample of 64 coordinates, skipping those whose argmin flips under +-h."""
    n, m, h = 2048, 128, 1e-6
    x = synth.random_walk(1 << 16, seed=58, dtype=np.float32)[:n].astype(np.float64)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    prof, pi = mp.matrix_profile(xt, m, 0.5, "fp64")
    loss = prof.sum() + prof.topk(16).values.mean()
    loss.backward()
    gx = xt.grad.cpu().numpy()
    mp0, pi0, _ = oracle.selfjoin(x, m)
    top0 = set(np.argsort(-mp0, kind="stable")[:16].tolist())

    def L(v):
        mpv, piv, _ = oracle.selfjoin(v, m)
        topv = np.argsort(-mpv, kind="stable")[:16]
        return mpv.sum() + mpv[topv].mean(), piv, set(topv.tolist())

    coords = np.sort(np.random.default_rng(59).choice(n, 64, replace=False))
    fd, keep = [], []
    for p in coords:
        xp, xm = x.copy(), x.copy()
        xp[p] += h
        xm[p] -= h
        lp, pip, tp = L(xp)
        lm, pim, tm = L(xm)
        if np.array_equal(pip, pi0) and np.array_equal(pim, pi0) and tp == top0 and tm == top0:
            fd.append((lp - lm) / (2 * h))
            keep.append(p)
    assert len(keep) >= 32
    fd = np.array(fd)
    err = np.linalg.norm(gx[keep] - fd) / np.linalg.norm(fd)
    assert err <= 1e-3, err
