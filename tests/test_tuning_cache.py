"""The binding's launch-shape cache (Context.autotune / Batch.autotune with a
JSON file): a miss times and stores the choice, a hit applies it without
timing, and the key separates GPUs, binnings, thresholds and sizes.  A fake
library stands in for the CUDA one (host logic only)."""
import ctypes
import json

import pytest

from paper_1507_03074_gb300 import ht


class FakeLib:
    def __init__(self):
        self.timed, self.applied = 0, []

    def ht_autotune(self, h, reps, t, us):
        self.timed += 1
        t._obj.fill_rows, t._obj.fill_threads, t._obj.fill_fused_scan = 32, 512, 1
        us._obj.value = 61.5
        return 0

    ht_batch_autotune = ht_autotune

    def ht_set_tuning(self, h, t):
        self.applied.append({n: int(getattr(t._obj, n)) for n in ht.TUNING_FIELDS})
        return 0

    ht_batch_set_tuning = ht_set_tuning

    def ht_destroy(self, h):
        return 0

    ht_batch_destroy = ht_destroy


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(ht, "lib", lambda: lib)
    monkeypatch.setattr(ht, "_gpu_name", lambda: "GB300-test")
    monkeypatch.delenv("HT_TUNING_CACHE", raising=False)
    return lib


class _Ctx:
    """A Context over the fake library whose handle is dropped after one
    autotune call, so that no later destructor reaches the real library."""

    def __init__(self, binning, threshold=10, max_hits=5000):
        self.binning, self.threshold, self.max_hits = binning, threshold, max_hits

    def autotune(self, **kw):
        c = object.__new__(ht.Context)
        c.binning, c.ranges, c.threshold, c.max_hits = self.binning, ht.Ranges(), self.threshold, self.max_hits
        c._h = ctypes.c_void_p(1)
        try:
            return c.autotune(**kw)
        finally:
            c._h = ctypes.c_void_p()


_ctx = _Ctx


def test_miss_then_hit(fake, tmp_path):
    path = str(tmp_path / "tuning.json")
    b = ht.Binning(4, 16, 1024, 1024)
    t1, us1 = _ctx(b).autotune(cache=path)
    assert fake.timed == 1 and not fake.applied and us1 == 61.5
    t2, us2 = _ctx(b).autotune(cache=path)
    assert fake.timed == 1                     # no second timing
    assert fake.applied == [t1] and t2 == t1 and us2 == us1
    d = json.load(open(path))
    key = next(iter(d))
    assert len(d) == 1 and key.startswith(f"GB300-test|k{ht._kernel_build_id()}|context|4x16x1024x1024")


def test_key_separates_configurations(fake, tmp_path, monkeypatch):
    path = str(tmp_path / "tuning.json")
    b = ht.Binning(4, 16, 1024, 1024)
    _ctx(b).autotune(cache=path)
    _ctx(ht.Binning(8, 32, 2048, 2048)).autotune(cache=path)
    _ctx(b, threshold=12).autotune(cache=path)
    _ctx(b, max_hits=50000).autotune(cache=path)
    monkeypatch.setattr(ht, "_gpu_name", lambda: "another GPU")
    _ctx(b).autotune(cache=path)
    # other kernel sources: a shape timed with the old kernels is not reused
    monkeypatch.setattr(ht, "_kernel_build_id", lambda: "changed")
    _ctx(b).autotune(cache=path)
    assert fake.timed == 6 and len(json.load(open(path))) == 6


def test_env_default_and_no_cache(fake, tmp_path, monkeypatch):
    b = ht.Binning(2, 4, 64, 64)
    _ctx(b).autotune()
    _ctx(b).autotune()
    assert fake.timed == 2                     # no cache without a path
    path = str(tmp_path / "env.json")
    monkeypatch.setenv("HT_TUNING_CACHE", path)
    _ctx(b).autotune()
    _ctx(b).autotune()
    assert fake.timed == 3 and len(fake.applied) == 1


def test_bad_cache_is_a_miss(fake, tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text("not json")
    b = ht.Binning(4, 16, 1024, 1024)
    _ctx(b).autotune(cache=str(path))
    assert fake.timed == 1
    key = next(iter(json.load(open(path))))
    path.write_text(json.dumps({key: {"tuning": {"no_such_field": 1}, "us_per_event": 1.0}}))
    _ctx(b).autotune(cache=str(path))
    assert fake.timed == 2                     # unknown fields: timed again


def test_batch_cache(fake, tmp_path):
    path = str(tmp_path / "tuning.json")
    B = object.__new__(ht.Batch)
    B.binning, B.ranges, B.threshold, B.max_events, B.max_hits = ht.Binning(4, 16, 1024, 1024), ht.Ranges(), 10, 100, 1 << 20
    B._h = ctypes.c_void_p(1)
    try:
        B.autotune(cache=path)
        B.autotune(cache=path)
    finally:
        B._h = ctypes.c_void_p()
    assert fake.timed == 1 and len(fake.applied) == 1
    assert "|batch|" in next(iter(json.load(open(path))))


def test_refused_cached_shape_is_retuned(fake, tmp_path, monkeypatch):
    """A cached shape that the library refuses (HT_E_INVAL from set_tuning)
    is timed again instead of raising."""
    path = str(tmp_path / "tuning.json")
    b = ht.Binning(4, 16, 1024, 1024)
    _ctx(b).autotune(cache=path)
    monkeypatch.setattr(fake, "ht_set_tuning", lambda h, t: ht.HT_E_INVAL, raising=False)
    monkeypatch.setattr(ht, "last_error", lambda: "refused")
    t, us = _ctx(b).autotune(cache=path)
    assert fake.timed == 2 and us == 61.5
