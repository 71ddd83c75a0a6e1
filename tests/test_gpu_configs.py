"""GPU parity at the full workload sizes (sampled rows, checked one by one
against the oracle), in the launch configurations the library uses by
default:

* AB-join of a 2^21 random walk against a 2^19 white-noise / random-walk
  mix with ten flat stretches of 2m, m = 512, both directions, in both
  precisions: 4,096 rows of A, 4,096 rows of B plus every row near a flat
  stretch's transitions; the join symmetry A-B vs B-A; and the FP32-mixed
  path at the autotuner's most extreme tile configuration (32,768-row tiles,
  no re-anchoring), where its error bias is widest;
* 4,096 ragged random walks (lengths 1000..65536, m in {32, 64, 128}) in one
  batched launch, in both precisions: 64 series, every row of the short ones
  and 256 rows of the others;
* the pan profile of a 2^16 random walk over 64 geometric window sizes
  16..1024, in both precisions: 128 rows at every size;
* the gradient of sum(MP) + mean(top-16 MP) on a 2^16 series, m = 128,
  against the oracle's closed form at the oracle's own argmin pairs, and
  against FP64 central differences of the oracle's MP on a 2048-sample slice
  (256 coordinates) through both forward precisions.
"""
import math

import numpy as np
import pytest

import _golden
import oracle
from paper_1904_12626_gb300 import synth

from _parity import GAP, check_rows

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
def ab():
    """Inputs and the oracle's answers on the sampled rows of both sides."""
    a, b, flats, m = _golden.c3_inputs()
    (ra, rb), _ = _golden.c3_oracle(a, b, flats, m)
    return a, b, flats, m, ra, rb


def _check_ab(ab, ma, pa, mb, pb, tol):
    a, b, flats, m, ra, rb = ab
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    check_rows(a64, m, ra[0], ma, pa, *ra[1:], tol, y=b64)
    check_rows(b64, m, rb[0], mb, pb, *rb[1:], tol, y=a64)
    for s in flats:                                # fully flat windows: closed form
        assert mb[s + 1] == math.sqrt(2 * m) and pb[s + 1] == 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_abjoin_full_size_sampled(mp, ab, prec):
    a, b, flats, m, ra, rb = ab
    assert len(ra[0]) == 4096 and len(rb[0]) >= 4096 + 300
    out = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec=prec, check_status=True))
    _check_ab(ab, *out, TOL[prec])


@pytest.mark.parametrize("variant", [0, 7])
def test_abjoin_extreme_tiles_fp32(mp, ab, variant):
    """The FP32-mixed path certifies its neighbours with an error bias that is
    widest after a drop in the windows' norms (the white-noise blocks of B
    after random-walk ones) and grows with the rows walked since an anchor:
    32,768-row tiles without re-anchoring are the autotuner's extreme."""
    a, b, flats, m, ra, rb = ab
    out = (t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec="fp32", tile_rows=32768,
                                               anchor_every=0, variant=variant,
                                               check_status=True))
    _check_ab(ab, *out, TOL["fp32"])


def _same_or_tied(x, y, m, p1, p2, tol):
    """Rows where two runs chose different neighbours must be ties: the two
    neighbours' distances (by the oracle's definition) within `tol`."""
    for r in np.nonzero(p1 != p2)[0]:
        d1 = oracle.distance_ab(x, y, m, int(r), int(p1[r]))
        d2 = oracle.distance_ab(x, y, m, int(r), int(p2[r]))
        assert abs(d1 - d2) <= tol, f"row {r}: neighbours {p1[r]} / {p2[r]} at {d1} / {d2}"


def test_abjoin_symmetry_full_size(mp, ab):
    """A-B and B-A are the same join seen from both sides: the B side of the
    first is the A side of the second.  PI is identical wherever the two
    neighbours are not tied within the PI criterion's gap; on sampled rows both
    runs pass the oracle check, and MP agrees to FP64 rounding on equal pairs."""
    a, b, flats, m, ra, rb = ab
    res1 = [t.cpu().numpy() for t in mp.abjoin(_t(a), _t(b), m, prec="fp32")]
    res2 = [t.cpu().numpy() for t in mp.abjoin(_t(b), _t(a), m, prec="fp32")]
    ma, pa, mb, pb = res1
    ma2, pa2, mb2, pb2 = res2
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    _check_ab(ab, mb2, pb2, ma2, pa2, TOL["fp32"])   # the B-A run, its sides swapped
    for m1, p1, m2, p2, x, y in ((mb, pb, ma2, pa2, b64, a64), (ma, pa, mb2, pb2, a64, b64)):
        eq = p1 == p2
        assert eq.mean() > 0.999
        assert float(np.max(np.abs(m1[eq] - m2[eq]))) <= 1e-9
        _same_or_tied(x, y, m, p1, p2, GAP)


@pytest.fixture(scope="module")
def batch():
    """4,096 ragged walks and the oracle's answers on 64 seeded series: every
    row of a series with at most 4,096 windows, 256 seeded rows otherwise."""
    values, offsets, ms = synth.ragged_batch(4096, seed=55)
    rng = np.random.default_rng(56)
    series = np.sort(rng.choice(len(ms), 64, replace=False))
    short = [int(b) for b in range(len(ms))
             if int(offsets[b + 1] - offsets[b]) - int(ms[b]) + 1 <= 4096]
    if not any(int(offsets[b + 1] - offsets[b]) - int(ms[b]) + 1 <= 4096 for b in series):
        series = np.sort(np.append(series[:-1], short[0]))
    answers = []
    for b in series:
        n_b = int(offsets[b + 1] - offsets[b])
        m = int(ms[b])
        l = n_b - m + 1
        rows = synth.sample_rows(l, 256 if l > 4096 else l, seed=int(b))
        xb = values[offsets[b]:offsets[b + 1]].astype(np.float64)
        answers.append((int(b), m, rows, *oracle.selfjoin(xb, m, rows=rows)))
    return values, offsets, ms, answers


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_4096_ragged_sampled(mp, batch, prec):
    values, offsets, ms, answers = batch
    g_mp, g_pi, _ = mp.batched(_t(values), _t(offsets), _t(ms), prec=prec, check_status=True)
    g_mp, g_pi = g_mp.cpu().numpy(), g_pi.cpu().numpy()
    assert len(answers) == 64 and any(len(r) == int(offsets[b + 1] - offsets[b]) - m + 1
                                      for b, m, r, *_ in answers)
    for b, m, rows, mo, po, so in answers:
        xb = values[offsets[b]:offsets[b + 1]].astype(np.float64)
        o = int(offsets[b])
        l = len(xb) - m + 1
        check_rows(xb, m, rows, g_mp[o:o + l], g_pi[o:o + l], mo, po, so, TOL[prec],
                   excl=oracle.exclusion_zone(m))


@pytest.fixture(scope="module")
def pan_case():
    """A 2^16 walk, the 64 window sizes, and the oracle on 128 rows per size."""
    n = 1 << 16
    x = synth.random_walk(n, seed=57, dtype=np.float32)
    ms = synth.pan_windows()
    x64 = x.astype(np.float64)
    answers = []
    for k, m in enumerate(ms.tolist()):
        rows = synth.sample_rows(n - m + 1, 128, seed=k)
        answers.append((rows, *oracle.selfjoin(x64, m, rows=rows)))
    return x, ms, answers


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pan_64_sizes_sampled(mp, pan_case, prec):
    x, ms, answers = pan_case
    n = len(x)
    assert len(set(ms.tolist())) == 64 and ms[0] == 16 and ms[-1] == 1024
    pan, pi = mp.pan(_t(x), ms, prec=prec, check_status=True)
    pan, pi = pan.cpu().numpy(), pi.cpu().numpy()
    x64 = x.astype(np.float64)
    for k, (rows, mo, po, so) in enumerate(answers):
        m = int(ms[k])
        l = n - m + 1
        check_rows(x64, m, rows, pan[k, :l], pi[k, :l], mo, po, so, TOL[prec],
                   excl=oracle.exclusion_zone(m))
        assert np.isinf(pan[k, l:]).all() and (pi[k, l:] == -1).all()


def _loss_weights(mp_vals):
    """dL/dMP of L = sum(MP) + mean(top-16 MP)."""
    g = np.ones(len(mp_vals))
    g[np.argsort(-mp_vals, kind="stable")[:16]] += 1.0 / 16
    return g


def test_gradient_2p16(mp):
    """loss = sum(MP) + mean of the top-16 MP values on a 2^16 walk, m = 128.
    The oracle evaluates the closed-form gradient at its own argmin pairs and
    its own top 16.  Rows whose GPU and oracle neighbours differ must be ties
    (the oracle's best-to-second-best gap within 1e-3); the gradient is not
    defined there, so they get weight 0 on both sides."""
    n, m = 1 << 16, 128
    x_np = synth.random_walk(n, seed=58, dtype=np.float32)
    x64 = x_np.astype(np.float64)
    mo, po, so = oracle.selfjoin(x64, m)
    g = _loss_weights(mo)
    x = torch.tensor(x_np, device="cuda", requires_grad=True)
    prof, pi = mp.matrix_profile(x, m, 0.5, "fp32")
    pi = pi.cpu().numpy()
    assert set(np.argsort(-prof.detach().cpu().numpy(), kind="stable")[:16]) == \
        set(np.argsort(-mo, kind="stable")[:16])
    tie = pi != po
    assert (so[tie] - mo[tie] <= GAP).all(), "PI differs on a separated row"
    assert tie.mean() < 1e-3
    w = g.copy()
    w[tie] = 0.0
    loss = (prof.double() * torch.from_numpy(w).cuda()).sum()
    loss.backward()
    ref = oracle.grad(x64, m, po, w)
    gx = x.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(gx - ref) / np.linalg.norm(ref)
    assert err <= 1e-3, err


@pytest.fixture(scope="module")
def fd_case():
    """FP64 central differences (h = 1e-6) of the oracle's loss on the first
    2048 samples run as their own series, at 256 seeded coordinates; a
    coordinate whose perturbation changes any argmin pair or the top-16 set is
    left out (the loss is not differentiable there)."""
    n, m, h = 2048, 128, 1e-6
    x = synth.random_walk(1 << 16, seed=58, dtype=np.float32)[:n].astype(np.float64)
    mp0, pi0, _ = oracle.selfjoin(x, m)
    top0 = set(np.argsort(-mp0, kind="stable")[:16].tolist())

    def L(v):
        mpv, piv, _ = oracle.selfjoin(v, m)
        topv = np.argsort(-mpv, kind="stable")[:16]
        return mpv.sum() + mpv[topv].mean(), piv, set(topv.tolist())

    coords = np.sort(np.random.default_rng(59).choice(n, 256, replace=False))
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
    return x, m, pi0, _loss_weights(mp0), np.array(keep), np.array(fd)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gradient_central_differences_2048(mp, fd_case, prec):
    """The GPU gradient through each forward precision against FP64 central
    differences of the oracle's loss (256 coordinates, those where the loss
    is differentiable kept), and against the oracle's closed form at the
    oracle's own argmin pairs over all 2048 coordinates."""
    x, m, pi0, g0, keep, fd = fd_case
    assert len(keep) >= 128
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    prof, pi = mp.matrix_profile(xt, m, 0.5, prec)
    assert np.array_equal(pi.cpu().numpy(), pi0)
    loss = prof.sum() + prof.topk(16).values.mean()
    loss.backward()
    gx = xt.grad.cpu().numpy()
    err = np.linalg.norm(gx[keep] - fd) / np.linalg.norm(fd)
    assert err <= 1e-3, err
    ref = oracle.grad(x, m, pi0, g0)
    err = np.linalg.norm(gx - ref) / np.linalg.norm(ref)
    assert err <= 1e-9 if prec == "fp64" else err <= 1e-6, err
