"""Launch-shape autotuner for the single-lattice and batched steps.

Candidates (rows per z-segment, warps per block, row fetch) are timed with
CUDA events on the solver's own stream for a few steps each; the steps taken
while tuning are real time steps (results do not depend on the launch shape).
The best shape is applied and remembered in a JSON cache keyed by storage and
lattice size class.

For a batch of uneven lattices the candidates also include per-lattice
segment plans: every lattice's z-segments sized so that all work items hold
about the same number of rows and the items fill a chosen number of waves
of the warps that can be resident at once (segment_plan).
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


PLAN_WAVES = [1.0, 1.5, 2.0, 3.0, 4.0, 6.0]
PERSIST_WAVES = [0.9, 1.0]


def segment_plan(shapes: list, resident: int, waves: float, window: int = 64) -> list:
    """Rows per z-segment for each lattice (nr, nz) of a batch: the step's
    warp-rows (window-column windows x rows, summed over the lattices) split
    into about `waves` x `resident` work items of equal length, each lattice's
    rows cut into that many balanced segments."""
    warp_rows = sum(-(-nr // window) * nz for nr, nz in shapes)
    rows = max(1.0, warp_rows / max(1.0, waves * resident))
    plan = []
    for nr, nz in shapes:
        nseg = max(1, int(round(nz / rows)))
        plan.append(-(-nz // nseg))
    return plan


def _apply(batch, launch, waves, graph_steps):
    seg, wpb, fetch = launch
    batch.set_launch(seg, wpb, graph_steps, fetch)
    if waves:
        resident, _ = batch.occupancy()
        batch.set_segments(segment_plan([(s.nr, s.nz) for s in batch.solvers], resident, waves))
    else:
        batch.set_segments(None)


def _batch_key(batch) -> str:
    return f"batch/{batch.solvers[0].storage}/{_size_class(batch.nodes)}/{_size_class(len(batch.solvers))}"


def has_cached_batch_launch(batch, graph_steps: int = 50) -> bool:
    """Whether tune_batch would take this batch's launch from the cache (and
    so take no steps); applies that launch when it does."""
    with _lock:
        e = _load().get(_batch_key(batch))
    if not e or len(e.get("launch", [])) != 3 or "waves" not in e:
        return False
    _apply(batch, tuple(e["launch"]), e["waves"], graph_steps)
    resident, items = batch.occupancy()
    return e["launch"][2] != 5 or items <= resident


def tune_batch(batch, steps: int = 30, graph_steps: int = 50, use_cache: bool = True) -> tuple:
    """Pick the batch's launch: (seg_rows, warps_per_block, row_fetch) for
    every lattice, or a per-lattice segment plan (segment_plan) for a number
    of waves, with the TMA-ring step; keyed by storage, node count and
    lattice count.  Returns (seg_rows, warps_per_block, row_fetch, waves),
    waves = 0 for a common segment length."""
    key = _batch_key(batch)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache and len(cache[key].get("launch", [])) == 3 and "waves" in cache[key]:
        best = tuple(cache[key]["launch"]) + (cache[key]["waves"],)
        _apply(batch, best[:3], best[3], graph_steps)
        resident, items = batch.occupancy()
        if best[2] != 5 or items <= resident:
            return best
        # a persistent launch chosen for another batch of this size class
        # does not fit this one: tune it afresh
    plan_launches = [(4, 1, 3), (4, 2, 3)]
    if batch.solvers[0].storage == "fp32":  # three ring stages: 12 resident warps per SM instead of 10
        plan_launches += [(4, 1, 4), (4, 2, 4)]
    cands = [(c, 0.0) for c in BATCH_CANDIDATES] + [(c, w) for c in plan_launches for w in PLAN_WAVES]
    # one persistent launch per call: every item resident (at most one wave)
    cands += [((4, 2, 5), w) for w in PERSIST_WAVES]
    results = []
    for launch, waves in cands:
        _apply(batch, launch, waves, 0)
        if launch[2] == 5:
            resident, items = batch.occupancy()
            if items > resident:
                continue
        batch.step(2)
        results.append((_time(batch.stream, batch.step, steps), launch, waves))
    results.sort(key=lambda r: r[0])
    _, launch, waves = results[0]
    _apply(batch, launch, waves, graph_steps)
    with _lock:
        cache = _load()
        cache[key] = {"launch": list(launch), "waves": waves, "ms_per_step": results[0][0]}
        _store(cache)
    return tuple(launch) + (waves,)
