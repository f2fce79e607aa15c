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


def _round_binary32(x):
    """Exact rational -> nearest binary32 (ties to even), as an exact rational."""
    from fractions import Fraction
    if x == 0:
        return Fraction(0)
    s, a = (-1 if x < 0 else 1), abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    n, rem = divmod(m.numerator, m.denominator)
    if 2 * rem > m.denominator or (2 * rem == m.denominator and n % 2 == 1):
        n += 1
    return s * n * ulp


def test_u8_colour_conversion_rounds_like_ieee_division():
    """The kernels' 8-bit colour conversion (unit_from_u8: q = RN(x r) with
    r = RN(1/255), one exact FMA residual x - 255 q, then RN(q + residual r),
    Markstein's correction step) is the correctly rounded x / 255 for all 256
    inputs, in exact arithmetic; the plain product RN(x r) is not."""
    from fractions import Fraction
    import numpy as np
    r = _round_binary32(Fraction(1, 255))
    wrong_plain = 0
    for x in range(256):
        q = _round_binary32(x * r)
        e = x - 255 * q
        assert _round_binary32(e) == e                        # the FMA residual is exact
        ref = _round_binary32(Fraction(x, 255))
        assert _round_binary32(q + e * r) == ref, x
        assert float(ref) == float(np.float32(x) / np.float32(255))
        wrong_plain += q != ref
    assert wrong_plain > 0
