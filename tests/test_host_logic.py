"""Host-side logic that needs no GPU: the schedule autotuner's choice and its
cache (the candidate timing is replaced by a fake)."""
import json

import pytest

from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")


class _Map:
    n = 1_600_000


def _fake_timer(calls, slow_tile=(16, 16)):
    def time_candidate(m, frames_cams, exposure, targets, C, tile, sort_tile, rc, pc, steps):
        calls.append((tuple(tile), sort_tile))
        return 1.0 + 0.01 * sort_tile / 2048 + (0.05 if tuple(tile) == slow_tile else 0.0) + \
            (0.02 if tuple(tile) == (32, 8) else 0.0)
    return time_candidate


def test_cache_key_depends_on_shapes_classes_and_map_bucket():
    from paper_2405_14342_gb300 import autotune
    a = scenes.tiny_camera()
    b = scenes.make_camera(scenes.PERSP, 640, 360, 400.0, 400.0, scenes.look_rotation(0.0, 0.0), (0, 0, 1))
    k = autotune.cache_key([a, b], 19, 1_600_000)
    assert k == autotune.cache_key([b, a], 19, 1_600_000)           # order of views does not matter
    assert k == autotune.cache_key([a, b], 19, 2_000_000)           # same power-of-two bucket (2^21)
    assert k != autotune.cache_key([a, b], 19, 3_000_000)
    assert k != autotune.cache_key([a, b], 8, 1_600_000)
    assert k != autotune.cache_key([a, a, b], 19, 1_600_000)        # view count


def test_tune_picks_the_fastest_candidate_and_caches_it(tmp_path, monkeypatch):
    from paper_2405_14342_gb300 import autotune
    calls = []
    monkeypatch.setattr(autotune, "_time_candidate", _fake_timer(calls))
    cams = [scenes.tiny_camera()]
    path = str(tmp_path / "sub" / "tune.json")
    choice, timings = autotune.tune(_Map(), [cams], None, None, 19, 1, 1, cache_path=path)
    assert len(calls) == len(autotune.TILES) * len(autotune.SORT_TILES) == len(timings)
    assert choice == {"tile": (8, 8), "sort_tile": 2048}
    cached = json.load(open(path))
    assert list(cached.values())[0]["tile"] == [8, 8]
    # the same key comes from the cache without timing anything
    calls.clear()
    again, t2 = autotune.tune(_Map(), [cams], None, None, 19, 1, 1, cache_path=path)
    assert again == choice and not calls and t2 == timings
    # another class count is a new key: timed and added beside the first
    monkeypatch.setattr(autotune, "_time_candidate", _fake_timer(calls, slow_tile=(8, 8)))
    other, _ = autotune.tune(_Map(), [cams], None, None, 8, 1, 1, cache_path=path)
    assert calls and other == {"tile": (16, 16), "sort_tile": 2048}
    assert len(json.load(open(path))) == 2
