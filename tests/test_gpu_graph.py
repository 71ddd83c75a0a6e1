"""Every join is a fixed sequence of kernels and memsets on the caller's
stream with no host synchronisation and no allocation, so it can be recorded
in a CUDA graph once and replayed; the replay must give the eager results,
also after the input is overwritten in place."""
import numpy as np
import pytest

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


def test_selfjoin_graph_replay(mp):
    import ctypes

    from paper_1904_12626_gb300 import _lib
    n, m = 20000, 64
    x = torch.from_numpy(synth.random_walk(n, seed=81)).cuda()
    cfg = _lib.make_config(m, 0.5, "fp32")
    ws = mp.workspace(_lib.load().mp_selfjoin_workspace_bytes(n, ctypes.byref(cfg)), x.device)
    a0, b0 = mp.selfjoin(x, m, ws=ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        a, b = mp.selfjoin(x, m, ws=ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, a0) and torch.equal(b, b0)
    x.copy_(torch.from_numpy(synth.random_walk(n, seed=82)).cuda())
    a1, b1 = mp.selfjoin(x, m, ws=ws)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, a1) and torch.equal(b, b1)
    assert not torch.equal(a1, a0)


def test_batched_graph_replay(mp):
    values, offsets, ms = synth.ragged_batch(64, seed=83, len_lo=1000, len_hi=4000)
    v = torch.from_numpy(values).cuda()
    o = torch.from_numpy(offsets).cuda()
    mm = torch.from_numpy(ms).cuda()
    max_m = int(ms.max())
    a0, b0, _ = mp.batched(v, o, mm, max_m=max_m)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        a, b, _ = mp.batched(v, o, mm, max_m=max_m)
    g.replay()
    torch.cuda.synchronize()
    used = np.zeros(len(values), bool)            # slots [o_b, o_b + l_b) of each series
    for k in range(len(ms)):
        used[offsets[k]:offsets[k + 1] - ms[k] + 1] = True
    used = torch.from_numpy(used).cuda()
    assert torch.equal(a[used], a0[used]) and torch.equal(b[used], b0[used])
