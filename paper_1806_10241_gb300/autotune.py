"""Launch-shape autotuner for the single-lattice and batched steps.

Candidates (rows per z-segment, warps per block, row fetch) are timed with
CUDA events on the solver's own stream for a few steps each; the steps taken
while tuning are real time steps (results do not depend on the launch shape).
The best shape is applied and remembered in a JSON cache keyed by storage and
lattice size class.
"""
from __future__ import annotations

import json
import os
import threading

import torch

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_lock = threading.Lock()

SOLVER_CANDIDATES = [(4, 1, 3), (4, 2, 3), (6, 1, 3), (8, 1, 3), (12, 2, 3), (16, 4, 3),
                     (6, 1, 2), (8, 2, 2), (8, 2, 1), (16, 4, 1)]
BATCH_CANDIDATES = [(4, 1, 3), (4, 2, 3), (6, 1, 3), (8, 1, 3), (8, 2, 1), (16, 4, 1)]


def _size_class(n: int) -> int:
    return max(0, int(n - 1).bit_length())


def _load() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: dict) -> None:
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, _CACHE)


def _time(stream, fn, steps: int) -> float:
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_solver(solver, steps: int = 20, use_cache: bool = True) -> tuple:
    """Pick (seg_rows, warps_per_block, row_fetch) for this solver's shape."""
    key = f"solver/{solver.storage}/{_size_class(solver.nr)}/{_size_class(solver.nz)}"
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        best = tuple(cache[key]["launch"])
        solver.set_launch(*best)
        return best
    cands = SOLVER_CANDIDATES if solver.storage != "fp64" else [(s, w, 1) for s in (16, 32) for w in (2, 4)]
    results = []
    for c in cands:
        solver.set_launch(*c)
        solver.step(2)  # warm
        results.append((_time(solver.stream, solver.step, steps), c))
    results.sort()
    best = results[0][1]
    solver.set_launch(*best)
    with _lock:
        cache = _load()
        cache[key] = {"launch": list(best), "ms_per_step": results[0][0]}
        _store(cache)
    return best


def tune_batch(batch, steps: int = 10, graph_steps: int = 10, use_cache: bool = True) -> tuple:
    """Pick (seg_rows, warps_per_block, row_fetch) for a batch, keyed by its node count."""
    key = f"batch/{batch.solvers[0].storage}/{_size_class(batch.nodes)}/{_size_class(len(batch.solvers))}"
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache and len(cache[key]["launch"]) == 3:
        best = tuple(cache[key]["launch"])
        batch.set_launch(best[0], best[1], graph_steps, best[2])
        return best
    results = []
    for seg, wpb, fetch in BATCH_CANDIDATES:
        batch.set_launch(seg, wpb, 0, fetch)
        batch.step(2)
        results.append((_time(batch.stream, batch.step, steps), (seg, wpb, fetch)))
    results.sort()
    best = results[0][1]
    batch.set_launch(best[0], best[1], graph_steps, best[2])
    with _lock:
        cache = _load()
        cache[key] = {"launch": list(best), "ms_per_step": results[0][0]}
        _store(cache)
    return best
