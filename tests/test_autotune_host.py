"""The FFT autotuner's host logic on the CPU: candidate plans, the JSON cache."""
import json

from paper_2501_10622_gb300 import autotune


def test_factorisations_multiply_to_the_length():
    for n in (192, 350, 512, 27):
        fs = autotune.factorisations(n)
        assert fs and all(1 <= len(f) <= 3 for f in fs)
        for f in fs:
            prod = 1
            for r in f:
                prod *= r
                assert r in autotune.RADICES
            assert prod == n
    assert (32,) in autotune.factorisations(32) and (2, 16) in autotune.factorisations(32)
    assert autotune.factorisations(1150) == []  # 23 is no radix


def test_candidates_prefer_large_radices_and_cover_tiles():
    c = autotune.candidates(512, limit=4)
    assert len(c) == 16 and {t for t, _ in c} == set(autotune.TILES)
    assert min(c[0][1]) >= min(c[-1][1])


def test_cache_round_trip(tmp_path):
    plans = {96: {"ng": 96, "yz": [8, [12, 8]], "x": None}, 32: {"ng": 32, "yz": None, "x": [4, [16]]}}
    path = autotune.save(plans, tmp_path / "plans.json")
    assert json.loads(path.read_text())["96"]["yz"] == [8, [12, 8]]
    assert autotune.load(path) == plans


def test_apply_sets_every_cached_pass():
    calls = []

    class FakeCtx:
        def set_fft_plan(self, ng, which, C=0, radices=()):
            calls.append((ng, which, C, tuple(radices)))
            return True

    autotune.apply(FakeCtx(), {96: {"yz": [8, [12, 8]], "x": None}, 32: {"yz": None, "x": [4, [16]]}})
    assert sorted(calls) == [(32, 1, 4, (16,)), (96, 0, 8, (12, 8))]
