"""PyTorch-facing wrappers of the C ABI (argument marshalling only).

Tensors are CUDA tensors; PyTorch provides the device memory (outputs and
workspace) and the current stream, and every computation happens inside
libmpgb's kernels.  Names follow the paper: the matrix profile ``mp`` and the
profile index ``pi`` (Sec. 2), self-join / AB-join (Sec. 3.2), window size
``m`` and exclusion-zone fraction ``ez`` (the ``window_size`` and
``exclusion_zone`` arguments of Sec. 3.2).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import MP_F32, MP_F64, check, make_config

_DT = {torch.float32: MP_F32, torch.float64: MP_F64}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dtype(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise TypeError(f"series must be float32 or float64, got {t.dtype}")
    return _DT[t.dtype]


def _prep(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dim() != 1:
        raise ValueError(f"{name} must be 1-D")
    return x.contiguous()


def workspace(nbytes: int, device) -> torch.Tensor:
    """A caller-owned workspace (torch allocations are 512-byte aligned)."""
    if nbytes <= 0:
        raise ValueError("workspace query failed (invalid configuration)")
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


def init(device: int | None = None) -> None:
    d = torch.cuda.current_device() if device is None else int(device)
    check(_lib.load().mp_init(d), "mp_init")


def profile_length(n: int, m: int) -> int:
    return int(_lib.load().mp_profile_length(n, m))


def exclusion_zone(m: int, ez: float = 0.5) -> int:
    return int(_lib.load().mp_exclusion_zone(m, ez))


def stats(x: torch.Tensor, m: int, stream=None):
    """(mu, invn, df, dg, flat) per window (FP64; flat as uint8)."""
    x = _prep(x, "x")
    lib = _lib.load()
    n = x.numel()
    l = n - m + 1
    if l <= 0:
        raise ValueError("m > n")
    out = [torch.empty(l, dtype=torch.float64, device=x.device) for _ in range(4)]
    flat = torch.empty(l, dtype=torch.uint8, device=x.device)
    check(lib.mp_stats(x.data_ptr(), _dtype(x), n, m, *(o.data_ptr() for o in out),
                       flat.data_ptr(), _stream(stream)), "mp_stats")
    return (*out, flat)


def selfjoin(x: torch.Tensor, m: int, ez: float = 0.5, prec: str = "fp32", *, refine: bool = True,
             inclusive: bool = False, raw: bool = False, tile_rows: int = 0, anchor_every: int = 0,
             variant: int = -1, ws: torch.Tensor | None = None, stream=None,
             check_status: bool = False):
    """Self-join matrix profile of one series.  Returns (mp float64, pi int64).
    raw=True: the non-normalised distance ||x_i - x_j|| (SiMPle)."""
    x = _prep(x, "x")
    lib = _lib.load()
    flags = ((0 if refine else _lib.MP_FLAG_NO_REFINE) | (_lib.MP_FLAG_EXCL_INCLUSIVE if inclusive else 0)
             | (_lib.MP_FLAG_RAW if raw else 0))
    cfg = make_config(m, ez, prec, anchor_every, tile_rows, variant, flags)
    n = x.numel()
    l = n - m + 1
    if m < 4 or l < 1:
        raise ValueError("need 4 <= m <= n")
    need = lib.mp_selfjoin_workspace_bytes(n, ctypes.byref(cfg))
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    mp = torch.empty(l, dtype=torch.float64, device=x.device)
    pi = torch.empty(l, dtype=torch.int64, device=x.device)
    check(lib.mp_selfjoin(x.data_ptr(), _dtype(x), n, ctypes.byref(cfg), mp.data_ptr(), pi.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream(stream)), "mp_selfjoin")
    if check_status:
        device_status(ws, stream)
    return mp, pi


def selfjoin_lr(x: torch.Tensor, m: int, ez: float = 0.5, prec: str = "fp32", *,
                refine: bool = True, inclusive: bool = False, raw: bool = False,
                tile_rows: int = 0, anchor_every: int = 0, variant: int = -1,
                ws: torch.Tensor | None = None, stream=None, check_status: bool = False):
    """Left and right self-join profiles.  Returns (mp_left, pi_left, mp_right, pi_right):
    the nearest neighbour of each window among the windows before / after it."""
    x = _prep(x, "x")
    lib = _lib.load()
    flags = ((0 if refine else _lib.MP_FLAG_NO_REFINE) | (_lib.MP_FLAG_EXCL_INCLUSIVE if inclusive else 0)
             | (_lib.MP_FLAG_RAW if raw else 0))
    cfg = make_config(m, ez, prec, anchor_every, tile_rows, variant, flags)
    n = x.numel()
    l = n - m + 1
    if m < 4 or l < 1:
        raise ValueError("need 4 <= m <= n")
    need = lib.mp_selfjoin_lr_workspace_bytes(n, ctypes.byref(cfg))
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    out = [torch.empty(l, dtype=dt, device=x.device)
           for dt in (torch.float64, torch.int64, torch.float64, torch.int64)]
    check(lib.mp_selfjoin_lr(x.data_ptr(), _dtype(x), n, ctypes.byref(cfg),
                             *(t.data_ptr() for t in out), ws.data_ptr(), ws.numel(),
                             _stream(stream)), "mp_selfjoin_lr")
    if check_status:
        device_status(ws, stream)
    return tuple(out)


class Anytime:
    """Anytime self-join: bands of diagonals in a seeded random order, run a
    cumulative fraction at a time.  `run(f)` returns the best-so-far (mp, pi)."""

    def __init__(self, x: torch.Tensor, m: int, seed: int = 0, ez: float = 0.5,
                 prec: str = "fp32", *, variant: int = -1, tile_rows: int = 0, stream=None,
                 ws: torch.Tensor | None = None):
        self.x = _prep(x, "x")
        self.lib = _lib.load()
        self.cfg = make_config(m, ez, prec, 0, tile_rows, variant, 0)
        self.n = self.x.numel()
        self.l = self.n - m + 1
        if m < 4 or self.l < 1:
            raise ValueError("need 4 <= m <= n")
        self.stream = stream
        need = self.lib.mp_anytime_workspace_bytes(self.n, ctypes.byref(self.cfg))
        self.ws = ws if ws is not None and ws.numel() >= need else workspace(need, self.x.device)
        check(self.lib.mp_anytime_begin(self.x.data_ptr(), _dtype(self.x), self.n,
                                        ctypes.byref(self.cfg), int(seed) & (2**64 - 1),
                                        self.ws.data_ptr(), self.ws.numel(), _stream(stream)),
              "mp_anytime_begin")

    def run(self, fraction: float, check_status: bool = False):
        mp = torch.empty(self.l, dtype=torch.float64, device=self.x.device)
        pi = torch.empty(self.l, dtype=torch.int64, device=self.x.device)
        check(self.lib.mp_anytime_run(self.n, ctypes.byref(self.cfg), float(fraction),
                                      mp.data_ptr(), pi.data_ptr(), self.ws.data_ptr(),
                                      self.ws.numel(), _stream(self.stream)), "mp_anytime_run")
        if check_status:
            device_status(self.ws, self.stream)
        return mp, pi


def fluss(pi: torch.Tensor, m: int, num_segments: int = 2, *, edge: int | None = None,
          seg_excl: int | None = None, ws: torch.Tensor | None = None, stream=None,
          check_status: bool = False):
    """Semantic segmentation (FLUSS) from a self-join profile index.
    Returns (cac float64 [l], segments int64 [num_segments], -1 when none is left).
    edge and seg_excl default to 5 m."""
    if pi.dtype != torch.int64 or not pi.is_cuda:
        raise TypeError("pi must be an int64 CUDA tensor")
    pi = pi.contiguous()
    lib = _lib.load()
    l = pi.numel()
    edge = 5 * m if edge is None else edge
    seg_excl = 5 * m if seg_excl is None else seg_excl
    need = lib.mp_fluss_workspace_bytes(l)
    if need == 0:
        raise ValueError("bad profile length")
    if ws is None or ws.numel() < need:
        ws = workspace(need, pi.device)
    cac = torch.empty(l, dtype=torch.float64, device=pi.device)
    seg = torch.empty(max(num_segments, 1), dtype=torch.int64, device=pi.device)
    check(lib.mp_fluss(pi.data_ptr(), l, edge, num_segments, seg_excl, cac.data_ptr(),
                       seg.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "mp_fluss")
    if check_status:
        device_status(ws, stream)
    return cac, seg[:num_segments]


def abjoin(a: torch.Tensor, b: torch.Tensor, m: int, prec: str = "fp32", *, refine: bool = True,
           both: bool = True, raw: bool = False, tile_rows: int = 0, anchor_every: int = 0,
           variant: int = -1, ws: torch.Tensor | None = None, stream=None,
           check_status: bool = False):
    """AB-join.  Returns (mp_a, pi_a, mp_b, pi_b); the B side is None unless `both`."""
    a = _prep(a, "a")
    b = _prep(b, "b")
    if a.dtype != b.dtype:
        raise TypeError("a and b must share a dtype")
    lib = _lib.load()
    cfg = make_config(m, 0.5, prec, anchor_every, tile_rows, variant,
                      (0 if refine else _lib.MP_FLAG_NO_REFINE) | (_lib.MP_FLAG_RAW if raw else 0))
    na, nb = a.numel(), b.numel()
    la, lb = na - m + 1, nb - m + 1
    if m < 4 or la < 1 or lb < 1:
        raise ValueError("need 4 <= m <= len(a), len(b)")
    need = lib.mp_abjoin_workspace_bytes(na, nb, ctypes.byref(cfg))
    if ws is None or ws.numel() < need:
        ws = workspace(need, a.device)
    mp_a = torch.empty(la, dtype=torch.float64, device=a.device)
    pi_a = torch.empty(la, dtype=torch.int64, device=a.device)
    mp_b = torch.empty(lb, dtype=torch.float64, device=a.device) if both else None
    pi_b = torch.empty(lb, dtype=torch.int64, device=a.device) if both else None
    check(lib.mp_abjoin(a.data_ptr(), na, b.data_ptr(), nb, _dtype(a), ctypes.byref(cfg),
                        mp_a.data_ptr(), pi_a.data_ptr(), mp_b.data_ptr() if both else None,
                        pi_b.data_ptr() if both else None, ws.data_ptr(), ws.numel(),
                        _stream(stream)), "mp_abjoin")
    if check_status:
        device_status(ws, stream)
    return mp_a, pi_a, mp_b, pi_b


def batched(values: torch.Tensor, offsets: torch.Tensor, ms: torch.Tensor, ez: float = 0.5,
            prec: str = "fp32", *, refine: bool = True, tile_rows: int = 0, anchor_every: int = 0,
            variant: int = -1, out_offsets: torch.Tensor | None = None, max_m: int | None = None,
            ws: torch.Tensor | None = None, stream=None, check_status: bool = False):
    """Self-joins of B ragged series in one persistent launch.

    values: concatenated series (CUDA); offsets: int64 [B+1] (CUDA);
    ms: int32 [B] (CUDA).  Returns (mp, pi, out_offsets): series b's profile
    is mp[out_offsets[b]:out_offsets[b+1]] (by default out_offsets is
    `offsets`, so each series keeps n_b slots of which the first l_b are used).
    """
    values = _prep(values, "values")
    lib = _lib.load()
    B = ms.numel()
    offsets = offsets.to(device=values.device, dtype=torch.int64).contiguous()
    ms = ms.to(device=values.device, dtype=torch.int32).contiguous()
    if out_offsets is None:
        out_offsets = offsets
    out_offsets = out_offsets.to(device=values.device, dtype=torch.int64).contiguous()
    if max_m is None:
        max_m = int(ms.max().item())
    cfg = make_config(4, ez, prec, anchor_every, tile_rows, variant,
                      0 if refine else _lib.MP_FLAG_NO_REFINE)
    total = values.numel()
    need = lib.mp_batched_workspace_bytes(total, B, max_m, ctypes.byref(cfg))
    if ws is None or ws.numel() < need:
        ws = workspace(need, values.device)
    nout = int(out_offsets[-1].item()) if out_offsets is not offsets else total
    mp = torch.empty(nout, dtype=torch.float64, device=values.device)
    pi = torch.empty(nout, dtype=torch.int64, device=values.device)
    check(lib.mp_batched(values.data_ptr(), _dtype(values), total, offsets.data_ptr(), ms.data_ptr(),
                         B, int(max_m), ctypes.byref(cfg), mp.data_ptr(), pi.data_ptr(),
                         out_offsets.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)),
          "mp_batched")
    if check_status:
        device_status(ws, stream)
    return mp, pi, out_offsets


def pan(x: torch.Tensor, ms, ez: float = 0.5, prec: str = "fp32", *, refine: bool = True,
        normalize: bool = False, tile_rows: int = 0, anchor_every: int = 0, variant: int = -1,
        ws: torch.Tensor | None = None, stream=None, check_status: bool = False):
    """Pan matrix profile over window sizes `ms` (host ints).  Returns
    (pan [nm x (n - min(ms) + 1)] float64, pi int64), +inf / -1 padded."""
    x = _prep(x, "x")
    lib = _lib.load()
    ms = [int(v) for v in ms]
    nm = len(ms)
    arr = (ctypes.c_int32 * nm)(*ms)
    flags = (0 if refine else _lib.MP_FLAG_NO_REFINE) | (_lib.MP_FLAG_PAN_NORMALIZE if normalize else 0)
    cfg = make_config(min(ms), ez, prec, anchor_every, tile_rows, variant, flags)
    n = x.numel()
    need = lib.mp_pan_workspace_bytes(n, arr, nm, ctypes.byref(cfg))
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    width = n - min(ms) + 1
    out = torch.empty((nm, width), dtype=torch.float64, device=x.device)
    pi = torch.empty((nm, width), dtype=torch.int64, device=x.device)
    check(lib.mp_pan(x.data_ptr(), _dtype(x), n, arr, nm, ctypes.byref(cfg), out.data_ptr(),
                     pi.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "mp_pan")
    if check_status:
        device_status(ws, stream)
    return out, pi


def backward(x: torch.Tensor, m: int, pi: torch.Tensor, grad_mp: torch.Tensor,
             ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """d(sum_i grad_mp[i] MP_i)/dx with the argmin pairs (i, pi[i]) fixed (FP64)."""
    x = _prep(x, "x")
    lib = _lib.load()
    n = x.numel()
    pi = pi.to(dtype=torch.int64).contiguous()
    g = grad_mp.to(dtype=torch.float64).contiguous()
    need = lib.mp_backward_workspace_bytes(n, m)
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    gx = torch.empty(n, dtype=torch.float64, device=x.device)
    check(lib.mp_backward(x.data_ptr(), _dtype(x), n, m, pi.data_ptr(), g.data_ptr(), gx.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream(stream)), "mp_backward")
    return gx


def device_status(ws: torch.Tensor, stream=None) -> None:
    """Synchronise and raise if the calls that used `ws` recorded a device error."""
    check(_lib.load().mp_get_device_status(ws.data_ptr(), _stream(stream)), "device status")


class MatrixProfileFn(torch.autograd.Function):
    """Differentiable self-join MP: forward = mp_selfjoin, backward = mp_backward.

    The gradient holds each row's argmin pair fixed (the MP is piecewise
    smooth in x; at ties it is a subgradient)."""

    @staticmethod
    def forward(ctx, x, m, ez=0.5, prec="fp32"):
        mp, pi = selfjoin(x.detach(), m, ez, prec)
        ctx.save_for_backward(x.detach(), pi)
        ctx.m = m
        ctx.mark_non_differentiable(pi)
        return mp.to(x.dtype), pi

    @staticmethod
    def backward(ctx, grad_mp, grad_pi):  # noqa: ARG004 - pi has no gradient
        x, pi = ctx.saved_tensors
        gx = backward(x, ctx.m, pi, grad_mp)
        return gx.to(x.dtype), None, None, None


def matrix_profile(x: torch.Tensor, m: int, ez: float = 0.5, prec: str = "fp32"):
    """Autograd-aware self-join: returns (mp, pi)."""
    return MatrixProfileFn.apply(x, m, ez, prec)
