"""Autotuner of a join's tile configuration.

Three knobs set how fast a join runs and never what it returns:

* the tile shape, ``variant``: one compiled instantiation of the
  diagonal-tile kernel (diagonals per band x rows per staged chunk x warps
  per CTA; ``mp_variant_count`` / ``mp_variant_info``);
* the row-tile height, ``tile_rows``: the rows one ticket of the work queue
  walks down its band, so the queue's granularity and the distance between
  exact FP64 anchors (0: the library's choice, which shortens the default
  height for small joins so that the persistent grid stays balanced);
* the re-anchor interval K, ``anchor_every``: further exact FP64 anchors
  inside a tile (the exact first dot product, then reuse, of STOMP,
  Sec. 3.3.2).  A shorter interval narrows the error bound the FP32
  recurrence carries, so fewer cells are replayed and compared exactly, at
  the price of m FP64 multiply-adds per diagonal per anchor.

Which setting is fastest depends on the family (self, left/right, AB,
batched, pan), the window, the sizes and the device, so the tuner measures
instead of guessing.  It times candidates on the caller's input with CUDA
events on the current stream, in three stages:

1. every variant at the library's tile height and no extra anchors;
2. the two fastest variants at each tile height of the precision's ladder;
3. the fastest pair at K = tile height / 2, / 4, / 8 (the default height's
   fractions when the library's height won; the library drops an interval
   not shorter than the height it runs).

It keeps the fastest candidate whose output agrees with the default
configuration's within the precision's error budget (``|dMP| <= 1e-3`` for
the FP32-mixed path, ``1e-9`` for FP64, with the same rows without a
neighbour; the FP32-mixed path certifies its neighbours exactly, so there
its outputs are in fact identical), and caches the choice as JSON, keyed by
family, precision, distance, window, size bucket (powers of two) and device.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import tempfile
import warnings
from dataclasses import asdict, dataclass
from typing import Callable, Iterable, Sequence

import torch

CACHE_VERSION = 1
TOL = {"fp32": 1e-3, "fp64": 1e-9}
TILE_ROWS = {"fp32": (1024, 2048, 4096, 8192, 16384, 32768), "fp64": (1024, 2048, 4096, 8192)}
DEFAULT_TILE_ROWS = {"fp32": 16384, "fp64": 4096}   # the library's defaults
DEFAULT_TILE_ROWS_AB_FP32 = 2048                     # FP32-mixed AB-joins (shorter tiles)
ANCHOR_DIVISORS = (2, 4, 8)
TOP_VARIANTS = 2


@dataclass(frozen=True)
class Candidate:
    """One tile configuration, in the library's resolved form (tile_rows and
    anchor_every whole multiples of the variant's chunk rows; tile_rows 0 =
    the library's choice; anchor_every 0 = no extra anchors)."""
    variant: int
    tile_rows: int
    anchor_every: int

    def kwargs(self) -> dict:
        return {"variant": self.variant, "tile_rows": self.tile_rows,
                "anchor_every": self.anchor_every}


def _ceil_to(v: int, q: int) -> int:
    return -(-v // q) * q


def resolve(variant: int, chunk_rows: int, tile_rows: int, anchor_every: int) -> Candidate:
    """The configuration the library runs for these arguments: both lengths
    rounded up to whole chunks; an interval not shorter than the tile means
    anchors at tile starts only (with tile_rows 0 the library settles the
    height, and that rule, per call)."""
    k = _ceil_to(anchor_every, chunk_rows) if anchor_every > 0 else 0
    if tile_rows <= 0:
        return Candidate(variant, 0, k)
    tr = _ceil_to(tile_rows, chunk_rows)
    return Candidate(variant, tr, 0 if k >= tr else k)


@dataclass
class Space:
    """Candidates of one tuning problem: the variants (with their chunk rows)
    and the precision's tile-height ladder."""
    variants: Sequence[tuple[int, int]]          # (variant, chunk_rows)
    tile_rows: Sequence[int]
    default_tile_rows: int

    def chunk_rows(self, variant: int) -> int:
        return dict(self.variants)[variant]

    def stage1(self) -> list[Candidate]:
        return _unique(resolve(v, rc, 0, 0) for v, rc in self.variants)

    def stage2(self, variants: Iterable[int]) -> list[Candidate]:
        return _unique(resolve(v, self.chunk_rows(v), tr, 0)
                       for v in variants for tr in self.tile_rows)

    def stage3(self, best: Candidate) -> list[Candidate]:
        rc = self.chunk_rows(best.variant)
        tr = best.tile_rows or self.default_tile_rows
        return _unique(resolve(best.variant, rc, best.tile_rows, tr // d)
                       for d in ANCHOR_DIVISORS if tr // d >= rc)


def _unique(cands: Iterable[Candidate]) -> list[Candidate]:
    out: list[Candidate] = []
    for c in cands:
        if c not in out:
            out.append(c)
    return out


def staged_search(space: Space, measure: Callable[[Candidate], float | None]
                  ) -> tuple[Candidate, dict[Candidate, float | None]]:
    """The three stages above.  `measure` returns a candidate's time in ms,
    or None when it is rejected (unsupported here, or its output disagrees);
    each candidate is measured once.  The default configuration (variant 0
    at the library's height) is measured first and is the answer when
    nothing else is faster; ties go to the earlier-measured candidate."""
    times: dict[Candidate, float | None] = {}

    def timed(c: Candidate) -> float | None:
        if c not in times:
            times[c] = measure(c)
        return times[c]

    def ranked(cands: Iterable[Candidate]) -> list[Candidate]:
        ok = [c for c in _unique(cands) if timed(c) is not None]
        return sorted(ok, key=lambda c: (times[c], list(times).index(c)))

    default = resolve(space.variants[0][0], space.variants[0][1], 0, 0)
    if timed(default) is None:
        raise RuntimeError("the default tile configuration was rejected")
    s1 = ranked([default] + space.stage1())
    s2 = ranked(s1[:1] + space.stage2(c.variant for c in s1[:TOP_VARIANTS]))
    s3 = ranked(s2[:1] + space.stage3(s2[0]))
    return s3[0], times


def outputs_agree(ref: Sequence[torch.Tensor], out: Sequence[torch.Tensor], tol: float) -> bool:
    """(mp, pi, mp, pi, ...) tuples agree within the error budget: the same
    rows without a neighbour (+inf / -1) and |dMP| <= tol elsewhere.  A
    different index on a row is allowed only where the distances agree,
    i.e. on a tie within the budget."""
    if len(ref) != len(out):
        return False
    for k in range(0, len(ref), 2):
        a, b = ref[k], out[k]
        pa, pb = ref[k + 1], out[k + 1]
        if a.shape != b.shape or pa.shape != pb.shape:
            return False
        if not torch.equal(torch.isinf(a), torch.isinf(b)) or not torch.equal(pa < 0, pb < 0):
            return False
        if torch.isnan(a).any() or torch.isnan(b).any():
            return False
        fin = torch.isfinite(a)
        if fin.any() and float((a[fin] - b[fin]).abs().max()) > tol:
            return False
    return True


def time_cuda_ms(fn: Callable[[], object], warmup: int, reps: int) -> float:
    """Median elapsed time of `fn` over `reps` runs (after `warmup` runs),
    from CUDA events on the current stream, synchronised on both sides."""
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def size_bucket(*sizes: int) -> str:
    """Sizes to the next power of two (a tuned choice holds within a bucket)."""
    return "x".join(f"2^{max(0, math.ceil(math.log2(max(1, int(s)))))}" for s in sizes)


def device_id() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


def cache_key(family: str, prec: str, raw: bool, m: int, sizes: Sequence[int], device: str) -> str:
    return "|".join([family, prec, "raw" if raw else "znorm", f"m{int(m)}", size_bucket(*sizes),
                     device])


@dataclass
class Choice:
    """A tuned configuration and the evidence for it."""
    variant: int
    tile_rows: int
    anchor_every: int
    ms: float
    default_ms: float
    measured: int

    def kwargs(self) -> dict:
        return {"variant": self.variant, "tile_rows": self.tile_rows,
                "anchor_every": self.anchor_every}


class Tuner:
    """Chooses and caches tile configurations.

    Each family method returns keyword arguments (``variant``, ``tile_rows``,
    ``anchor_every``) for the matching ``api`` call, e.g.::

        tuner = Tuner("mpgb_tune.json")
        mp, pi = api.selfjoin(x, m, **tuner.selfjoin(x, m))

    A cached key is answered without running anything.  ``cache_path=None``
    keeps the cache in memory only.
    """

    def __init__(self, cache_path: str | os.PathLike | None = None, *, warmup: int = 1,
                 reps: int = 3, timer: Callable[[Callable[[], object], int, int], float] | None = None,
                 space_fn: Callable[[str, bool], Space] | None = None,
                 device: str | None = None):
        self.cache_path = os.fspath(cache_path) if cache_path is not None else None
        self.warmup, self.reps = int(warmup), int(reps)
        self._timer = timer or time_cuda_ms
        self._space_fn = space_fn or library_space
        self._device = device
        self.entries: dict[str, dict] = {}
        self.measured = 0                        # candidates timed by this tuner
        self.last: Choice | None = None          # the most recent answer
        if self.cache_path and os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as f:
                    data = json.load(f)
                if data.get("version") == CACHE_VERSION and isinstance(data.get("entries"), dict):
                    self.entries = data["entries"]
                else:
                    warnings.warn(f"{self.cache_path}: not a version-{CACHE_VERSION} tuning cache; "
                                  "starting empty")
            except (OSError, ValueError) as e:
                warnings.warn(f"{self.cache_path}: unreadable tuning cache ({e}); starting empty")

    # -- generic ---------------------------------------------------------
    def tune(self, key: str, prec: str, raw: bool, run: Callable[[Candidate], Sequence[torch.Tensor]],
             default_tile_rows: int | None = None) -> Choice:
        """Answer `key` from the cache, else search with `run` (which runs
        the join with a candidate and returns its (mp, pi, ...) outputs)."""
        if key in self.entries:
            try:
                self.last = Choice(**self.entries[key])
                return self.last
            except TypeError:
                warnings.warn(f"tuning cache entry {key!r} is malformed; tuning again")
        from ._lib import MPError
        space = self._space_fn(prec, raw)
        if default_tile_rows:
            space = Space(space.variants, space.tile_rows, default_tile_rows)
        tol = TOL[prec]
        ref: list[Sequence[torch.Tensor]] = []

        def measure(c: Candidate) -> float | None:
            try:
                out = run(c)
                if not ref:
                    ref.append(out)
                elif not outputs_agree(ref[0], out, tol):
                    return None
                self.measured += 1
                return self._timer(lambda: run(c), self.warmup, self.reps)
            except MPError:
                return None

        best, times = staged_search(space, measure)
        default = next(iter(times))
        ch = Choice(best.variant, best.tile_rows, best.anchor_every, float(times[best]),
                    float(times[default]), sum(t is not None for t in times.values()))
        self.entries[key] = asdict(ch)
        self.save()
        self.last = ch
        return ch

    def save(self) -> None:
        if not self.cache_path:
            return
        d = os.path.dirname(os.path.abspath(self.cache_path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump({"version": CACHE_VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def _key(self, family, prec, raw, m, sizes):
        return cache_key(family, prec, raw, m, sizes, self._device or device_id())

    # -- families ----------------------------------------------------------
    def selfjoin(self, x: torch.Tensor, m: int, ez: float = 0.5, prec: str = "fp32", *,
                 raw: bool = False, inclusive: bool = False) -> dict:
        from . import api
        key = self._key("self", prec, raw, m, [x.numel()])
        return self.tune(key, prec, raw, lambda c: api.selfjoin(
            x, m, ez, prec, raw=raw, inclusive=inclusive, **c.kwargs())).kwargs()

    def selfjoin_lr(self, x: torch.Tensor, m: int, ez: float = 0.5, prec: str = "fp32", *,
                    raw: bool = False, inclusive: bool = False) -> dict:
        from . import api
        key = self._key("lr", prec, raw, m, [x.numel()])
        return self.tune(key, prec, raw, lambda c: api.selfjoin_lr(
            x, m, ez, prec, raw=raw, inclusive=inclusive, **c.kwargs())).kwargs()

    def abjoin(self, a: torch.Tensor, b: torch.Tensor, m: int, prec: str = "fp32", *,
               raw: bool = False) -> dict:
        from . import api
        key = self._key("ab", prec, raw, m, [a.numel(), b.numel()])
        return self.tune(key, prec, raw, lambda c: api.abjoin(
            a, b, m, prec, raw=raw, **c.kwargs()),
            default_tile_rows=DEFAULT_TILE_ROWS_AB_FP32 if prec == "fp32" else None).kwargs()

    def batched(self, values: torch.Tensor, offsets: torch.Tensor, ms: torch.Tensor,
                ez: float = 0.5, prec: str = "fp32", *, max_m: int | None = None) -> dict:
        from . import api
        off = offsets.to(device=values.device, dtype=torch.int64)
        mm = ms.to(device=values.device, dtype=torch.int64)
        if max_m is None:
            max_m = int(mm.max().item())
        # compact outputs (no unused slots) so that candidates compare element-wise
        lens = torch.clamp(off[1:] - off[:-1] - mm + 1, min=0)
        out_off = torch.cat([lens.new_zeros(1), torch.cumsum(lens, 0)])
        key = self._key("batched", prec, False, max_m, [values.numel(), ms.numel()])

        def run(c):
            mp, pi, _ = api.batched(values, off, ms, ez, prec, out_offsets=out_off, max_m=max_m,
                                    **c.kwargs())
            return mp, pi
        return self.tune(key, prec, False, run).kwargs()

    def pan(self, x: torch.Tensor, ms, ez: float = 0.5, prec: str = "fp32") -> dict:
        from . import api
        ms = [int(v) for v in ms]
        key = self._key("pan", prec, False, min(ms), [x.numel(), len(ms), max(ms)])
        return self.tune(key, prec, False,
                         lambda c: api.pan(x, ms, ez, prec, **c.kwargs())).kwargs()


def library_space(prec: str, raw: bool) -> Space:
    """The candidates the loaded library offers for a precision (the
    non-normalised distance is compiled for variant 0 only)."""
    import ctypes

    from . import _lib
    lib = _lib.load()
    pid = 1 if prec == "fp32" else 0
    variants = []
    for v in range(1 if raw else int(lib.mp_variant_count(pid))):
        td, rc = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(lib.mp_variant_info(pid, v, ctypes.byref(td), ctypes.byref(rc)), "mp_variant_info")
        variants.append((v, rc.value))
    return Space(variants, TILE_ROWS[prec], DEFAULT_TILE_ROWS[prec])
