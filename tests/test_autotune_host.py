"""Host-side logic of the autotuner (no GPU): size classes and the persisted
table, with the timing step replaced by a stub."""
import json

import numpy as np
import pytest

autotune = pytest.importorskip("paper_1405_7958_gb300.autotune")


class _Img:
    def __init__(self, H, W):
        self.shape = (H, W)


def test_size_class_buckets_count_and_megapixels():
    assert autotune.size_class([_Img(4096, 4096)] * 8) == "n8_mp128"
    assert autotune.size_class([_Img(1024, 1024), _Img(1024, 3072)]) == "n2_mp4"
    assert autotune.size_class([_Img(1000, 1000)]) == autotune.size_class([_Img(1010, 1000)])


def test_table_tunes_once_per_class_and_persists(tmp_path, monkeypatch):
    calls = []

    def fake_tune(images, **kw):
        calls.append(autotune.size_class(images))
        return {"best": {"variant": 1, "max_local": 8 + len(calls), "strip_tiles": 4 * len(calls), "ms": 1.0},
                "all": []}

    monkeypatch.setattr(autotune, "tune", fake_tune)
    path = tmp_path / "table.json"
    t = autotune.Table(str(path))
    a = [_Img(2048, 2048)] * 3
    b = [_Img(4096, 4096)]
    p1 = t.params(a)
    p2 = t.params(a)
    p3 = t.params(b)
    assert calls == ["n3_mp12", "n1_mp16"]            # each class tuned once
    assert (p1.variant, p1.max_local, p1.strip_tiles) == (p2.variant, p2.max_local, p2.strip_tiles) == (1, 9, 4)
    assert (p3.max_local, p3.strip_tiles) == (10, 8)
    stored = json.loads(path.read_text())
    assert set(stored) == {"n3_mp12", "n1_mp16"}
    t2 = autotune.Table(str(path))                    # a new table reads the file: no tuning
    assert t2.params(b).max_local == 10 and len(calls) == 2


def test_candidates_cover_schedules_and_strips():
    vs = {v for v, _, _ in autotune.CANDIDATES}
    assert vs == {autotune.rt.RT_RASTER, autotune.rt.RT_HYBRID, autotune.rt.RT_FRONTIER}
    assert all(m >= 0 and 0 <= st <= 32 for _, m, st in autotune.CANDIDATES)
    raster = [(m, st) for v, m, st in autotune.CANDIDATES if v == autotune.rt.RT_RASTER]
    assert len({st for _, st in raster}) > 1 and len({m for m, _ in raster}) > 1


def test_old_tables_without_a_strip_still_load(tmp_path):
    path = tmp_path / "old.json"
    path.write_text(json.dumps({"n1_mp16": {"variant": 1, "max_local": 12, "ms": 1.0}}))
    p = autotune.Table(str(path)).params([_Img(4096, 4096)])
    assert (p.variant, p.max_local, p.strip_tiles) == (1, 12, 0)
