"""Continuous-batching server of axisymmetric solve requests.

Requests (workloads.Request: arrival time + lattice) arrive as a stream.  The
server keeps every admitted lattice resident on the device and advances all
of them together with the batched step (one persistent launch per step,
replayed from a CUDA graph).  Between rounds it
  * admits the requests that have arrived while their bytes fit the device
    memory budget (lb_required_bytes against free HBM less a reserve) and,
    when node_budget is set, while the nodes being stepped stay within it
    (a lone request is always admitted): once the resident lattices fill
    the GPU, more of them only lengthen every active request's latency
    without raising the update rate, so the rest wait in arrival order,
  * evaluates the diagnostics of each active lattice every `check_every`
    steps and retires the ones that reached the steady state
    (|Nu(t) - Nu(t - window)| < tol), hit the step cap or diverged,
  * rebuilds the batch when its membership changed (with autotune, a new
    size class is tuned on scratch copies of the lattices, so that the
    live ones are checked at the same steps as in a solo run).
A request whose lattice can never fit the budget is rejected; `cancel(rid)`
withdraws a request (pending: dropped; active: retired at the end of the
round).  Latency of a request = finish time - arrival time.
`run_sequential` serves the same stream one plain solve at a time, for
comparison.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from .autotune import has_cached_batch_launch, tune_batch
from .batch import Batch
from .solver import Solver, required_bytes
from .workloads import Request


@dataclass
class Record:
    rid: int
    name: str
    nodes: int
    arrival: float
    admitted: float = -1.0
    finished: float = -1.0
    steps: int = 0
    nu: float = float("nan")
    status: str = "pending"  # converged | capped | diverged | rejected | cancelled

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class Report:
    records: list
    makespan: float
    mode: str
    extra: dict = field(default_factory=dict)

    def summary(self) -> dict:
        done = [r for r in self.records if r.finished >= 0]
        solved = [r for r in done if r.status in ("converged", "capped", "diverged")]
        lat = np.array([r.latency for r in solved]) if solved else np.array([np.nan])
        ok = [r for r in done if r.status == "converged"]
        steps_nodes = sum(r.steps * r.nodes for r in solved)
        return {"mode": self.mode, "requests": len(self.records), "completed": len(done),
                "converged": len(ok), "capped": sum(r.status == "capped" for r in done),
                "diverged": sum(r.status == "diverged" for r in done),
                "rejected": sum(r.status == "rejected" for r in done),
                "cancelled": sum(r.status == "cancelled" for r in done),
                "makespan_s": round(self.makespan, 3),
                "solves_per_s": round(len(solved) / self.makespan, 3) if self.makespan > 0 else None,
                "p50_latency_s": round(float(np.percentile(lat, 50)), 3),
                "p99_latency_s": round(float(np.percentile(lat, 99)), 3),
                "MLUPS": round(steps_nodes / self.makespan / 1e6, 1) if self.makespan > 0 else None,
                **self.extra}


class _Active:
    def __init__(self, req: Request, solver: Solver, rec: Record, nbytes: int):
        self.req, self.solver, self.rec, self.nbytes = req, solver, rec, nbytes
        self.history: list[tuple[int, float]] = []  # (step, Nu)
        self.last_check = 0  # step of the last diagnostics


def _steady(history: list[tuple[int, float]], window: int, tol: float) -> bool:
    if len(history) < 2:
        return False
    s_now, nu_now = history[-1]
    for s, nu in reversed(history[:-1]):
        if s_now - s >= window:
            return abs(nu_now - nu) < tol
    return False


class Server:
    def __init__(self, storage: str = "fp16", steps_per_round: int = 500, check_every: int = 500,
                 window: int = 1000, tol: float = 1e-6, max_steps: int = 200_000,
                 hbm_budget: int | None = None, reserve_bytes: int = 1 << 30, max_active: int = 512,
                 graph_steps: int = 50, seg_rows: int = 0, warps_per_block: int = 0,
                 device: str = "cuda", keep_results: bool = False, autotune: bool = False,
                 node_budget: int | None = None):
        if check_every % steps_per_round:
            raise ValueError("check_every must be a multiple of steps_per_round")
        self.storage = storage
        self.steps_per_round = steps_per_round
        self.check_every = check_every
        self.window = window
        self.tol = tol
        self.max_steps = max_steps
        self.max_active = max_active
        self.node_budget = node_budget
        self.max_nodes = 0  # most nodes stepped together
        self.graph_steps = graph_steps
        self.seg_rows = seg_rows
        self.warps_per_block = warps_per_block
        self.autotune = autotune
        self.device = torch.device(device)
        self.keep_results = keep_results
        self.results: dict[int, np.ndarray] = {}  # final distributions (keep_results)
        self.max_concurrent = 0
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = (free - reserve_bytes) if hbm_budget is None else int(hbm_budget)
        self.stream = torch.cuda.Stream(self.device)
        self._cancelled: set[int] = set()

    def cancel(self, rid: int) -> None:
        """Withdraw request rid (takes effect at the next round boundary)."""
        self._cancelled.add(rid)

    # -- one request's admission and retirement ---------------------------------------
    def _admit(self, req: Request, now: float, rec: Record) -> _Active:
        s = Solver(req.case.params, storage=self.storage, device=self.device, stream=self.stream)
        s.init_fields(req.case.fields)
        rec.admitted = now
        return _Active(req, s, rec, required_bytes(req.case.params, self.storage))

    def _tune(self, batch: Batch, active: list, used: int) -> None:
        """The batch's launch from the autotuner (cached per storage and size
        class).  On a cache miss the candidates are timed on scratch copies
        of the active lattices, so that the live ones take no extra steps:
        their steady-state checks then fall on the same steps as in a solo
        run, and so do the results.  Only when the copies would not fit the
        memory budget are the live lattices tuned (the tuning steps are
        real steps)."""
        if not has_cached_batch_launch(batch, self.graph_steps) and 2 * used <= self.budget:
            scratch = []
            for a in active:
                s = Solver(a.req.case.params, storage=self.storage, device=self.device, stream=self.stream)
                s.init_fields(a.req.case.fields)
                scratch.append(s)
            sb = Batch(scratch, stream=self.stream, seg_rows=self.seg_rows, warps_per_block=self.warps_per_block,
                       graph_steps=self.graph_steps)
            tune_batch(sb, steps=3, graph_steps=self.graph_steps)
            sb.close()
            for s in scratch:
                s.close()
        tune_batch(batch, steps=3, graph_steps=self.graph_steps)

    def _check(self, a: _Active, d: dict | None = None) -> bool:
        """Diagnostics of an active lattice (given, or computed here); True
        when it is finished."""
        if d is None:
            d = a.solver.diag()
        a.last_check = d["step"]
        a.rec.steps = d["step"]
        a.rec.nu = d["nu_avg"]
        a.history.append((d["step"], d["nu_avg"]))
        if d["status"] != 0 or not np.isfinite(d["nu_avg"]):
            a.rec.status = "diverged"
            return True
        if _steady(a.history, self.window, self.tol):
            a.rec.status = "converged"
            return True
        if d["step"] >= self.max_steps:
            a.rec.status = "capped"
            return True
        return False

    def run(self, requests: list[Request], clock=time.perf_counter, on_round=None) -> Report:
        """Serve the stream; on_round(server, now) is called after every round."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        records = {r.rid: Record(r.rid, r.case.name, r.case.nr * r.case.nz, r.arrival) for r in requests}
        active: list[_Active] = []
        used = 0
        nodes = 0
        batch = None
        dirty = True
        t0 = clock()
        rounds = 0
        while pending or active:
            now = clock() - t0
            # withdrawn requests that are still waiting
            if self._cancelled and pending:
                keep = deque()
                for req in pending:
                    if req.rid in self._cancelled:
                        rec = records[req.rid]
                        rec.status, rec.finished = "cancelled", now
                    else:
                        keep.append(req)
                pending = keep
            # admit what has arrived, in arrival order, while it fits
            while pending and pending[0].arrival <= now and len(active) < self.max_active:
                need = required_bytes(pending[0].case.params, self.storage)
                if need > self.budget:  # can never fit: reject
                    req = pending.popleft()
                    rec = records[req.rid]
                    rec.status, rec.finished = "rejected", clock() - t0
                    continue
                if used + need > self.budget:
                    break
                n_req = pending[0].case.nr * pending[0].case.nz
                if self.node_budget and active and nodes + n_req > self.node_budget:
                    break
                req = pending.popleft()
                active.append(self._admit(req, now, records[req.rid]))
                used += active[-1].nbytes
                nodes += n_req
                self.max_concurrent = max(self.max_concurrent, len(active))
                self.max_nodes = max(self.max_nodes, nodes)
                dirty = True
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival - (clock() - t0))))
                continue
            if dirty:
                if batch is not None:
                    batch.close()
                batch = Batch([a.solver for a in active], stream=self.stream, seg_rows=self.seg_rows,
                              warps_per_block=self.warps_per_block, graph_steps=self.graph_steps)
                if self.autotune:
                    self._tune(batch, active, used)
                dirty = False
            batch.step(self.steps_per_round)
            rounds += 1
            # diagnostics of the lattices whose last check is check_every steps back
            if on_round is not None:
                on_round(self, clock() - t0)
            finished = []
            due = [a.solver.step_count - a.last_check >= self.check_every for a in active]
            diags = batch.diag() if any(due) else None  # every lattice's diagnostics in one download
            for a, is_due, d in zip(active, due, diags or [None] * len(active)):
                if a.rec.rid in self._cancelled:
                    a.rec.steps = a.solver.step_count
                    a.rec.status = "cancelled"
                    finished.append(a)
                elif is_due and self._check(a, d):
                    finished.append(a)
            if finished:
                now = clock() - t0
                for a in finished:
                    a.rec.finished = now
                    if self.keep_results:
                        self.results[a.rec.rid] = a.solver.get_dist()
                    used -= a.nbytes
                    nodes -= a.rec.nodes
                    active.remove(a)
                    a.solver.close()
                batch.close()
                batch = None
                dirty = True
        if batch is not None:
            batch.close()
        torch.cuda.synchronize(self.device)
        return Report(list(records.values()), clock() - t0, "batched",
                      {"rounds": rounds, "storage": self.storage, "max_concurrent": self.max_concurrent,
                       "max_nodes": self.max_nodes, "node_budget": self.node_budget})

    def run_sequential(self, requests: list[Request], storage: str = "fp32",
                       clock=time.perf_counter) -> Report:
        """The same stream served one plain solve at a time (no batching)."""
        queue = deque(sorted(requests, key=lambda r: r.arrival))
        records = {r.rid: Record(r.rid, r.case.name, r.case.nr * r.case.nz, r.arrival) for r in requests}
        t0 = clock()
        while queue:
            req = queue.popleft()
            now = clock() - t0
            if req.arrival > now:
                time.sleep(req.arrival - now)
            rec = records[req.rid]
            s = Solver(req.case.params, storage=storage, device=self.device, stream=self.stream)
            s.init_fields(req.case.fields)
            a = _Active(req, s, rec, 0)
            rec.admitted = clock() - t0
            while True:
                s.step(self.steps_per_round)
                if s.step_count - a.last_check >= self.check_every and self._check(a):
                    break
            rec.finished = clock() - t0
            s.close()
        torch.cuda.synchronize(self.device)
        return Report(list(records.values()), clock() - t0, "sequential", {"storage": storage})
