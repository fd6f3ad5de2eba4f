"""Host logic of the autotuner cache (no GPU)."""
import json

from paper_2202_12477_gb300 import autotune as at
from paper_2202_12477_gb300 import hb


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    assert at.load(path) == {}
    dev = at.device_key("NVIDIA GB300", 152)
    c = at.record({}, dev, 7, hb.HB_F64, 3, {0: 12.9, 3: 12.5})
    at.record(c, dev, 7, hb.HB_F32, 7, {3: 1.48, 7: 1.45})
    at.record(c, dev, 7, hb.HB_F64X, 67, {3: 7.1, 67: 6.4})
    at.store(c, path)
    c2 = at.load(path)
    assert at.lookup(c2, dev, 7, hb.HB_F64) == 3
    assert at.lookup(c2, dev, 7, hb.HB_F32) == 7
    assert at.lookup(c2, dev, 7, hb.HB_F64X) == 67
    assert at.lookup(c2, dev, 9, hb.HB_F64) is None
    assert at.lookup(c2, at.device_key("other", 80), 7, hb.HB_F64) is None


def test_cache_rejects_garbage(tmp_path):
    path = tmp_path / "c.json"
    path.write_text("not json")
    assert at.load(str(path)) == {}
    dev = at.device_key("g", 1)
    path.write_text(json.dumps({dev: {at.entry_key(3, hb.HB_F64): {"variant": 6}}}))
    assert at.lookup(at.load(str(path)), dev, 3, hb.HB_F64) is None  # 6 is not a valid variant
    # the double-float kernel is not built in the EB2 shape
    path.write_text(json.dumps({dev: {at.entry_key(3, hb.HB_F64X): {"variant": 7}}}))
    assert at.lookup(at.load(str(path)), dev, 3, hb.HB_F64X) is None


def test_env_override(monkeypatch, tmp_path):
    monkeypatch.setenv("HB_AUTOTUNE_CACHE", str(tmp_path / "x.json"))
    assert at.cache_path() == str(tmp_path / "x.json")


def test_general_mesh_choice_leaves_out_the_lattice_gather(tmp_path):
    # the lattice-gather variants (GRID bit) rely on the box's structure; a
    # choice that must hold on any mesh takes the fastest of the others
    timings = {3: 12.5, 75: 12.3, 131: 12.1, 139: 12.2}
    assert at.best_allowed(timings, hb.HB_VARIANT_GRID) == 75
    assert at.best_allowed(timings, 0) == 131
    dev = at.device_key("NVIDIA GB300", 152)
    c = at.record({}, dev, 7, hb.HB_F64, 131, timings)
    at.record(c, dev, 7, hb.HB_F64, 75, timings, exclude=hb.HB_VARIANT_GRID)
    assert at.lookup(c, dev, 7, hb.HB_F64) == 131
    assert at.lookup(c, dev, 7, hb.HB_F64, exclude=hb.HB_VARIANT_GRID) == 75
    # a stored entry that breaks its own exclusion is not trusted
    c[dev][at.entry_key(7, hb.HB_F64, hb.HB_VARIANT_GRID)]["variant"] = 139
    assert at.lookup(c, dev, 7, hb.HB_F64, exclude=hb.HB_VARIANT_GRID) is None
