"""Host logic of the launch autotuner: size classes and the JSON cache (a
cached choice is applied without timing anything)."""
import json

from paper_1806_10241_gb300 import autotune


class FakeSolver:
    def __init__(self, storage, nr, nz):
        self.storage, self.nr, self.nz = storage, nr, nz
        self.launches, self.steps = [], 0

    def set_launch(self, *a):
        self.launches.append(a)

    def step(self, n=1):
        self.steps += n


def test_size_classes_are_powers_of_two():
    assert [autotune._size_class(n) for n in (1, 2, 3, 4, 5, 1024, 1025)] == [0, 1, 2, 2, 3, 10, 11]


def test_cached_solver_launch_is_applied_without_timing(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "_CACHE", str(path))
    s = FakeSolver("fp16", 1000, 2000)
    key = f"solver/fp16/{autotune._size_class(1000)}/{autotune._size_class(2000)}"
    path.write_text(json.dumps({key: {"launch": [6, 2, 3], "ms_per_step": 0.05}}))
    assert autotune.tune_solver(s) == (6, 2, 3)
    assert s.launches == [(6, 2, 3)] and s.steps == 0
    # another size class misses the cache entry (it would time candidates)
    assert f"solver/fp16/{autotune._size_class(5000)}" not in path.read_text()


def test_cache_survives_a_corrupt_file(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "_CACHE", str(path))
    path.write_text("{not json")
    assert autotune._load() == {}
    autotune._store({"a": {"launch": [4, 1, 3]}})
    assert autotune._load() == {"a": {"launch": [4, 1, 3]}}


def test_segment_plan_balances_items_and_fills_the_waves():
    """Every lattice's segments differ by at most one row from the common
    item length, and the item count is close to waves x resident warps."""
    shapes = [(64 + 7 * m, (64 + 7 * m) * (1 + m % 2)) for m in range(40)]
    resident = 1520
    for waves in autotune.PLAN_WAVES:
        plan = autotune.segment_plan(shapes, resident, waves)
        assert len(plan) == len(shapes)
        items = sum(-(-nr // 64) * -(-nz // seg) for (nr, nz), seg in zip(shapes, plan))
        assert 0.8 * waves * resident <= items <= 1.25 * waves * resident, (waves, items)
        rows = [nz / -(-nz // seg) for (nr, nz), seg in zip(shapes, plan)]
        assert max(rows) / min(rows) < 1.6, (waves, min(rows), max(rows))
        for (nr, nz), seg in zip(shapes, plan):
            assert 1 <= seg <= nz
    # one lattice far smaller than the item length keeps a single segment
    assert autotune.segment_plan([(64, 8), (1024, 2048)], 152, 1.0)[0] == 8


class FakeBatch:
    """The Batch surface tune_batch uses, with a fixed occupancy."""

    def __init__(self, resident, items):
        self.solvers = [FakeSolver("fp32", 64, 64)]
        self.nodes = 4096
        self.resident, self.items = resident, items
        self.launches, self.segments, self.steps = [], [], 0
        self.stream = None

    def set_launch(self, *a):
        self.launches.append(a)

    def set_segments(self, seg):
        self.segments.append(seg)

    def occupancy(self):
        return self.resident, self.items

    def step(self, n=1):
        self.steps += n


def test_cached_persistent_batch_launch_is_rechecked(tmp_path, monkeypatch):
    """A cached persistent launch (row fetch 5) is applied only when every work
    item of this batch is resident; otherwise the batch is tuned afresh."""
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "_CACHE", str(path))
    key = f"batch/fp32/{autotune._size_class(4096)}/{autotune._size_class(1)}"
    path.write_text(json.dumps({key: {"launch": [4, 2, 5], "waves": 1.0, "ms_per_step": 0.01}}))
    fits = FakeBatch(resident=100, items=50)
    assert autotune.tune_batch(fits) == (4, 2, 5, 1.0) and fits.steps == 0
    timed = []
    monkeypatch.setattr(autotune, "_time", lambda stream, fn, steps: timed.append(1) or 1.0)
    too_many = FakeBatch(resident=100, items=150)
    best = autotune.tune_batch(too_many)
    assert timed and best[2] != 5  # tuned again, and no persistent candidate could run


def test_has_cached_batch_launch(tmp_path, monkeypatch):
    """The server asks whether a batch's launch is cached (then it takes no
    tuning steps): not without an entry, yes for a cached launch, and not
    for a cached persistent launch whose items are not all resident."""
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "_CACHE", str(path))
    b = FakeBatch(resident=100, items=50)
    assert not autotune.has_cached_batch_launch(b)
    key = f"batch/fp32/{autotune._size_class(4096)}/{autotune._size_class(1)}"
    path.write_text(json.dumps({key: {"launch": [4, 2, 4], "waves": 1.0, "ms_per_step": 0.01}}))
    assert autotune.has_cached_batch_launch(b) and b.launches[-1][:2] == (4, 2)
    path.write_text(json.dumps({key: {"launch": [4, 2, 5], "waves": 1.0, "ms_per_step": 0.01}}))
    assert autotune.has_cached_batch_launch(b)
    assert not autotune.has_cached_batch_launch(FakeBatch(resident=100, items=150))
    assert b.steps == 0
