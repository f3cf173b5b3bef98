"""CPU checks of the batch autotuner's host logic (no GPU): size classes, the
per-class plan and its rows, the refinement's candidates, the search with a
timing model in place of the GPU, and the cache (key, reuse, rows applied)."""
import json

from paper_1308_1464_gb300 import autotune as at


class FakeBatch:
    def __init__(self):
        self.rows = None
        self.set_calls = 0

    def set_tile_rows(self, rows):
        self.rows = list(rows)
        self.set_calls += 1


def test_classes_and_plans():
    assert [at.class_of(my) for my in (16, 23, 24, 47, 48, 95, 96, 191, 192, 256)] == \
        [0, 0, 1, 1, 2, 2, 3, 3, 4, 4]
    sizes = [(16, 16), (30, 200), (100, 40), (256, 256), (17, 90)]
    # rows capped at the patch height (never below 8)
    assert at.rows_from_plan([8, 16, 32, 64, 128], sizes) == [8, 128, 16, 128, 32]
    assert at.rows_from_plan([64] * 5, [(16, 5)]) == [8]
    # the plan of a global policy: the rows it gives each class's median height
    assert at.plan_from_policy(at.POLICIES["half"], sizes) == [8, 16, 32, 32, 64]
    assert at.plan_from_policy(at.POLICIES["rows32"], sizes) == [32] * 5


def test_refinement_candidates():
    sizes = [(16, 16), (30, 200), (100, 40), (256, 256), (17, 90)]
    trials = at.refinement_trials([16] * 5, sizes)
    # classes by decreasing cells: 256x256 (class 4), 30x200 (class 4) ... 16x16 last
    assert trials[0][0] == 4 and trials[-1][0] == 0
    # rows stop at the first value covering the tallest patch of the class
    assert [r for k, r in trials if k == 0] == [8, 16]
    assert [r for k, r in trials if k == 4] == [8, 16, 32, 64, 128, 256]
    assert {k for k, _ in trials} == {0, 1, 2, 4}     # class 3 is empty


def test_search_and_cache(tmp_path, monkeypatch):
    sizes = [(16, 16), (30, 200), (100, 40), (256, 256), (17, 90)] * 3

    def model(batch, rows, reset, nsteps, cfl, repeats):
        # a timing model: the current rows (as created: 32 everywhere)
        r = rows if rows is not None else [32] * len(sizes)
        batch.rows = list(r)
        # best: 16 rows for patches up to 100 high, 64 above
        return sum(abs(x - (16 if my <= 100 else 64)) for x, (_, my) in zip(r, sizes)) + 1.0

    monkeypatch.setattr(at, "_time", model)
    cache = tmp_path / "tune.json"
    b = FakeBatch()
    desc, timings = at.tune_batch(b, sizes, lambda: None, cache_path=str(cache), device_name="fake")
    want = [16 if my <= 100 else 64 for _, my in sizes]
    assert b.rows == want, (desc, b.rows)
    assert "refined" in desc and timings["as_created"] > min(timings.values())
    data = json.loads(cache.read_text())
    key = at.cache_key(sizes, "fake")
    assert data[key]["rows"] == want
    # the cache key: sizes in any order, the device, the tuner version
    assert at.cache_key(list(reversed(sizes)), "fake") == key
    assert at.cache_key(sizes, "other") != key
    # a second call reuses the cache: no timing, the rows applied once
    monkeypatch.setattr(at, "_time", lambda *a, **k: (_ for _ in ()).throw(AssertionError("timed")))
    b2 = FakeBatch()
    desc2, _ = at.tune_batch(b2, sizes, lambda: None, cache_path=str(cache), device_name="fake")
    assert b2.rows == want and b2.set_calls == 1 and desc2 == desc
