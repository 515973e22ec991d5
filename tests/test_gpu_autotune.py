"""Launch autotuner: picks a candidate launch, caches it per storage and
size class, and never changes the results (the launch shape is invisible in
the bits)."""
import numpy as np
import pytest

from paper_1806_10241_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()


@pytest.fixture
def cache(tmp_path, monkeypatch):
    from paper_1806_10241_gb300 import autotune
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "_CACHE", str(path))
    return path


def test_solver_tuning_is_cached_and_invisible_in_the_results(cache):
    import json
    from paper_1806_10241_gb300 import autotune
    from paper_1806_10241_gb300.solver import Solver
    c = W.swirling_cylinder(nr=200, nz=300, Re=300.0, Ra=1e4, amp=1e-3, seed=4)
    ref = Solver(c.params, storage="fp16")
    ref.init_fields(c.fields)
    tuned = Solver(c.params, storage="fp16")
    tuned.init_fields(c.fields)
    best = autotune.tune_solver(tuned, steps=3)
    assert best in autotune.SOLVER_CANDIDATES
    assert tuned.get_launch() == best
    entry = json.loads(cache.read_text())
    assert list(entry.values())[0]["launch"] == list(best)
    ref.step(tuned.step_count)  # tuning steps are real steps
    assert np.array_equal(ref.get_dist(), tuned.get_dist())
    again = Solver(c.params, storage="fp16")
    assert autotune.tune_solver(again) == best  # from the cache, no timing
    assert again.step_count == 0


def test_batch_tuning_is_cached(cache):
    from paper_1806_10241_gb300 import autotune
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    sols = []
    for cs in W.batched_instances(6, lo=32, hi=96):
        s = Solver(cs.params, storage="bf16", stream=stream)
        s.init_fields(cs.fields)
        sols.append(s)
    b = Batch(sols, stream=stream)
    best = autotune.tune_batch(b, steps=3, graph_steps=4)
    assert (best[3] == 0 and best[:3] in autotune.BATCH_CANDIDATES) or (
        best[3] in autotune.PLAN_WAVES and best[2] in (3, 4)) or (best[3] in autotune.PERSIST_WAVES and best[2] == 5)
    assert autotune.tune_batch(b, steps=3, graph_steps=4) == best
    b.step(8)
    assert all(d["status"] == 0 for d in b.diag())
    b.close()
