"""Host logic of the autotuner (no GPU): the library's rounding of tile
configurations, the staged search, the error-budget check and the JSON
cache, driven by a fake join and a fake clock."""
import json
import warnings

import pytest
import torch

from paper_1904_12626_gb300 import tune
from paper_1904_12626_gb300._lib import MPError, MP_EUNSUPPORTED
from paper_1904_12626_gb300.tune import Candidate, Space

# a library with four variants: chunk rows 512, 512, 256, 256
SPACE = Space([(0, 512), (1, 512), (2, 256), (3, 256)], (4096, 8192, 16384, 32768), 16384)


def test_resolve_rounds_like_the_library():
    assert tune.resolve(0, 512, 16384, 0) == Candidate(0, 16384, 0)
    assert tune.resolve(0, 512, 1000, 0) == Candidate(0, 1024, 0)        # up to whole chunks
    assert tune.resolve(2, 256, 4096, 300) == Candidate(2, 4096, 512)
    assert tune.resolve(0, 512, 4096, 4096) == Candidate(0, 4096, 0)     # K >= tile: tile starts only
    assert tune.resolve(0, 512, 4096, 3900) == Candidate(0, 4096, 0)     # rounds up to the tile
    assert tune.resolve(0, 512, 4096, 511) == Candidate(0, 4096, 512)
    # height 0: the library's own choice, the interval still in whole chunks
    assert tune.resolve(0, 512, 0, 0) == Candidate(0, 0, 0)
    assert tune.resolve(0, 512, 0, 3000) == Candidate(0, 0, 3072)


def test_stages_enumerate_distinct_candidates():
    assert SPACE.stage1() == [Candidate(v, 0, 0) for v in range(4)]
    s2 = SPACE.stage2([1, 3])
    assert len(s2) == 8 and len(set(s2)) == 8
    s3 = SPACE.stage3(Candidate(2, 4096, 0))
    assert s3 == [Candidate(2, 4096, 2048), Candidate(2, 4096, 1024), Candidate(2, 4096, 512)]
    # the library's height won: fractions of the default height
    assert SPACE.stage3(Candidate(1, 0, 0)) == [Candidate(1, 0, 8192), Candidate(1, 0, 4096),
                                                Candidate(1, 0, 2048)]
    # intervals shorter than a chunk are left out, equal ones merge
    small = Space([(0, 512)], (1024,), 1024)
    assert small.stage3(Candidate(0, 1024, 0)) == [Candidate(0, 1024, 512)]


def _cost(c: Candidate) -> float:
    """A separable cost with its minimum at variant 2, 8192 rows, K = 2048."""
    v = {0: 10.0, 1: 12.0, 2: 9.0, 3: 11.0}[c.variant]
    t = {0: 0.5, 4096: 1.0, 8192: 0.0, 16384: 0.5, 32768: 2.0}[c.tile_rows]
    k = {0: 0.3, 4096: 0.2, 2048: 0.0, 1024: 0.4}[c.anchor_every]
    return v + t + k


def test_staged_search_finds_separable_optimum():
    seen = []

    def measure(c):
        seen.append(c)
        return _cost(c)
    best, times = tune.staged_search(SPACE, measure)
    assert best == Candidate(2, 8192, 2048)
    assert len(seen) == len(set(seen))                  # each candidate timed once
    assert seen[0] == Candidate(0, 0, 0)                # the library's default first
    assert len(seen) <= 4 + 2 * 4 + 3
    # the second-best variant of stage 1 (0) was tried at every height
    assert {c.tile_rows for c in seen if c.variant == 0} == {0, 4096, 8192, 16384, 32768}
    assert not any(c.variant in (1, 3) and c.tile_rows != 0 for c in seen)


def test_staged_search_never_picks_rejected_and_keeps_default_on_ties():
    def measure(c):
        if c.variant == 2:
            return None                                 # unsupported / disagrees
        return 5.0
    best, times = tune.staged_search(SPACE, measure)
    assert best == Candidate(0, 0, 0)
    assert times[Candidate(2, 0, 0)] is None
    with pytest.raises(RuntimeError):
        tune.staged_search(SPACE, lambda c: None)


def test_outputs_agree_is_the_error_budget():
    mp = torch.tensor([1.0, 2.0, float("inf"), 0.5], dtype=torch.float64)
    pi = torch.tensor([3, 0, -1, 1])
    assert tune.outputs_agree((mp, pi), (mp.clone(), pi.clone()), 1e-3)
    assert tune.outputs_agree((mp, pi), (mp + torch.tensor([9e-4, 0, 0, 0]), pi), 1e-3)
    assert not tune.outputs_agree((mp, pi), (mp + torch.tensor([2e-3, 0, 0, 0]), pi), 1e-3)
    assert not tune.outputs_agree((mp, pi), (mp + torch.tensor([2e-9, 0, 0, 0]), pi), 1e-9)
    # a tie within the budget may pick another index
    assert tune.outputs_agree((mp, pi), (mp, torch.tensor([2, 0, -1, 1])), 1e-3)
    # a row that lost (or gained) its neighbour does not agree
    mp2 = mp.clone()
    mp2[2] = 3.0
    assert not tune.outputs_agree((mp, pi), (mp2, torch.tensor([3, 0, 5, 1])), 1e-3)
    nan = mp.clone()
    nan[0] = float("nan")
    assert not tune.outputs_agree((mp, pi), (nan, pi), 1e-3)
    assert not tune.outputs_agree((mp, pi), (mp[:3], pi[:3]), 1e-3)
    # both sides of an AB-join are checked
    assert not tune.outputs_agree((mp, pi, mp, pi), (mp, pi, mp + 1.0, pi), 1e-3)


def test_size_bucket_and_key():
    assert tune.size_bucket(1 << 20) == "2^20"
    assert tune.size_bucket((1 << 20) + 1) == "2^21"
    assert tune.size_bucket(1, 3000) == "2^0x2^12"
    k = tune.cache_key("self", "fp32", False, 256, [1 << 20], "GB300/152sm")
    assert k == "self|fp32|znorm|m256|2^20|GB300/152sm"
    assert tune.cache_key("self", "fp32", True, 256, [1 << 20], "d") != tune.cache_key(
        "self", "fp32", False, 256, [1 << 20], "d")


class FakeJoin:
    """A join whose outputs and times depend on the candidate: variant 3 is
    fastest but returns a wrong distance; variant 1 is unsupported."""

    def __init__(self):
        self.calls = 0
        self.current = None

    def run(self, c):
        self.calls += 1
        if c.variant == 1:
            raise MPError(MP_EUNSUPPORTED, "fake")
        self.current = c
        mp = torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64)
        if c.variant == 3:
            mp = mp + 0.1
        return mp, torch.tensor([2, 2, 0])

    def timer(self, fn, warmup, reps):
        for _ in range(warmup + reps):
            fn()
        return _cost(self.current)


def _tuner(path, fake):
    return tune.Tuner(path, timer=fake.timer, space_fn=lambda prec, raw: SPACE, device="fake/1sm")


def test_tuner_rejects_wrong_outputs_and_caches(tmp_path):
    path = tmp_path / "tune.json"
    fake = FakeJoin()
    t = _tuner(path, fake)
    ch = t.tune("k1", "fp32", False, fake.run)
    assert (ch.variant, ch.tile_rows, ch.anchor_every) == (2, 8192, 2048)   # not variant 3
    assert ch.ms == pytest.approx(_cost(Candidate(2, 8192, 2048)))
    assert ch.default_ms == pytest.approx(_cost(Candidate(0, 0, 0)))
    assert t.last == ch and t.measured == ch.measured > 0
    data = json.loads(path.read_text())
    assert data["version"] == tune.CACHE_VERSION and "k1" in data["entries"]
    # a new tuner answers from the file without running anything
    fake2 = FakeJoin()
    t2 = _tuner(path, fake2)
    assert t2.tune("k1", "fp32", False, fake2.run) == ch
    assert fake2.calls == 0 and t2.measured == 0
    # another key is tuned and both are kept
    t2.tune("k2", "fp32", False, fake2.run)
    assert set(json.loads(path.read_text())["entries"]) == {"k1", "k2"}


def test_tuner_survives_a_corrupt_cache(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    fake = FakeJoin()
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        t = _tuner(path, fake)
    assert any("unreadable" in str(x.message) for x in w)
    t.tune("k", "fp32", False, fake.run)
    assert "k" in json.loads(path.read_text())["entries"]
    # a malformed entry is tuned again
    data = json.loads(path.read_text())
    data["entries"]["k"] = {"variant": 0}
    path.write_text(json.dumps(data))
    fake2 = FakeJoin()
    with warnings.catch_warnings(record=True):
        warnings.simplefilter("always")
        ch = _tuner(path, fake2).tune("k", "fp32", False, fake2.run)
    assert fake2.calls > 0 and ch.variant == 2


def test_tuner_in_memory_only():
    fake = FakeJoin()
    t = tune.Tuner(None, timer=fake.timer, space_fn=lambda prec, raw: SPACE, device="x")
    t.tune("k", "fp64", False, fake.run)
    t.save()                                            # no path: nothing written
    assert "k" in t.entries
