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
