#!/usr/bin/env python3
"""Benchmark of the fused axisymmetric cascaded LB step on GB300.

Default workload: the swirling heated cylinder on a 1024 x 2048 meridian
grid (H/R = 2, lid speed 0.05, Re = 1000, Ra = 1e5, Pr = 0.7), FP32.  A
"step" is one time step of the whole method (stream + sources + three
cascaded collisions + boundaries) over the lattice.  The metric is MLUPS
(million node updates per second, each update covering f, g and h).

  python bench.py [--gpus N --steps K --warmup W] [--storage fp32|fp16|bf16|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

With N > 1 (torchrun) every rank advances its own replica of the lattice
(the method has no exchange between independent solves): weak scaling, one
barrier and a max over ranks around the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (3-field node updates/s) & HBM roofline fraction; served solves/s, p99"
L2_BYTES = 129e6  # GB300 L2
BYTES_PER_NODE = {"fp64": 304, "fp32": 152, "bf16": 76, "fp16": 76}
DTYPE = {"fp64": "f64", "fp32": "f32", "bf16": "f32 (bf16 storage)", "fp16": "f32 (fp16 storage)"}
PROFILE_JSON = os.path.join(ROOT, "profiles", "roofline_counters.json")


def workload_desc(nr, nz, storage):
    return (f"swirling heated cylinder {nr}x{nz} (H/R=2, lid u=0.05, Re=1000, Ra=1e5, Pr=0.7), "
            f"{storage} storage")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def kernel_source_hash():
    """Hash of the step kernels' sources and the nvcc flags they are built with."""
    from paper_1806_10241_gb300.build import FLAGS
    h = hashlib.sha256()
    for name in ("lb_kernels.cu", "lb_internal.h", "lb_pair.cuh"):
        with open(os.path.join(ROOT, "paper_1806_10241_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    h.update(" ".join(FLAGS).encode())
    return h.hexdigest()[:16]


def kernel_name(storage, row_fetch):
    """The step kernel a launch configuration runs."""
    if storage == "fp64":
        return "k_step64"
    return {1: "k_step2", 2: "k_step2_tma", 3: "k_step3_tma"}[row_fetch]


def counters_for(key, what="dram_bytes_per_launch"):
    """A per-launch counter (DRAM traffic, warp instructions) from the
    committed ncu summary, only while the kernel source and build flags still
    match the ones the counters were taken on."""
    try:
        with open(PROFILE_JSON) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(key)
    if not e or e.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return e.get(what)


def issue_roofline(key, ms_per_step, sm_mhz):
    """Warp instructions per launch (ncu smsp__inst_executed.sum, committed)
    against the issue ceiling: every SM's four schedulers issue at most one
    warp instruction per cycle, at the SM clock seen under load."""
    import torch
    inst = counters_for(key, "warp_instructions_per_launch")
    if inst is None or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    achieved = inst / (ms_per_step * 1e-3) / 1e9
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions_per_launch": inst,
            "peak_kind": f"{sms} SMs x 4 schedulers x 1 warp instruction per cycle x {sm_mhz:.0f} MHz"}


# ---- clocks -------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples every 200 ms in the background; keeps timestamps so
    the timed window can be cut out afterwards."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        win = [s for t, s in self.samples if t0 - 0.1 <= t <= t1 + 0.1]
        if not win and self.samples:  # short timed region: nearest samples
            mid = 0.5 * (t0 + t1)
            win = [min(self.samples, key=lambda ts: abs(ts[0] - mid))[1]]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(s[1]) for s in win) if v is not None)
        smax = max((num(s[2]) or 0) for s in win)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in win for k in range(4)
                          if len(s) > 5 + k and s[5 + k].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(win), "power_w_max": max((num(s[3]) or 0) for s in win)}


# ---- multi-rank timing ---------------------------------------------------------------

def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, nodes: int, steps: int, ms: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica of `nodes` nodes."""
    return world * nodes * steps / (ms * 1e3)


# ---- the CPU oracle ---------------------------------------------------------------

def oracle_mlups(nr, nz_full, budget_s, max_rows=None):
    """Time the FP64 oracle on the host cores on a cylinder of nr columns and
    as many rows of the same workload as fit the budget (one step at least)."""
    import oracle
    from paper_1806_10241_gb300 import workloads as W
    oracle.build()
    threads = oracle.get_threads()
    rows = min(nz_full, max(8, 64))
    c = W.config_cylinder(nr, rows)
    o = oracle.Oracle(c.params)
    o.init_fields(c.fields)
    t = time.perf_counter()
    o.step(1)
    dt = max(time.perf_counter() - t, 1e-6)
    rate = nr * rows / dt
    steps = max(1, int(budget_s * rate / (nr * rows)))
    if max_rows:
        steps = min(steps, max_rows)
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    return {"value": round(nr * rows * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": threads,
            "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps of a {nr}x{rows} slab of the {nr}x{nz_full} "
                      f"cylinder workload (same per-node work), {threads} OpenMP threads, "
                      f"{dt:.1f} s"}


def serving_measure(requests, nr_lo, nr_hi, max_steps, storage, node_budget=0):
    """A Poisson stream of solve requests (rate 50/s, seed 0) served by the
    continuous-batching server (autotuned batched launches, graphs of 50) and,
    for comparison, by sequential plain FP32 solves; both with the steady
    test |dNu| < 1e-6 over 1000 steps and the step cap max_steps."""
    import torch
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.serving import Server
    reqs = W.serving_requests(count=requests, rate=50.0, seed=0, nr_lo=nr_lo, nr_hi=nr_hi)
    kw = dict(steps_per_round=500, check_every=500, window=1000, tol=1e-6, max_steps=max_steps)
    srv = Server(storage=storage, graph_steps=50, autotune=True, node_budget=node_budget or None, **kw)
    rep_b = srv.run(reqs)
    rep_s = Server(storage=storage, **kw).run_sequential(reqs, storage="fp32")
    torch.cuda.synchronize()
    rb, seq = rep_b.summary(), rep_s.summary()
    # the served Nu of each request against its sequential FP32 solve
    nu_s = {r.rid: r.nu for r in rep_s.records}
    dnu = [abs(r.nu - nu_s[r.rid]) / abs(nu_s[r.rid]) for r in rep_b.records
           if r.finished >= 0 and nu_s.get(r.rid) not in (None, 0.0)]
    return {"solves_per_s": rb["solves_per_s"], "p50_latency_s": rb["p50_latency_s"],
            "p99_latency_s": rb["p99_latency_s"],
            "config": {"requests": requests, "rate_per_s": 50.0, "nr": f"U{{{nr_lo}..{nr_hi}}}",
                       "nz": "nr * U{1,2}", "Ra": "log-U[1e3,1e5]", "mix": "60 % annulus, 40 % cylinder",
                       "steady": "|dNu| < 1e-6 over 1000 steps", "max_steps": max_steps, "storage": storage,
                       "batch_launch": "autotuned per size class",
                       "admission": "free HBM" + (f" and at most {node_budget} nodes stepped together"
                                                  if node_budget else "")},
            "nu_rel_diff_vs_sequential_fp32": {"max": float(max(dnu)) if dnu else None,
                                               "median": float(sorted(dnu)[len(dnu) // 2]) if dnu else None},
            "batched": rb, "sequential_fp32": seq,
            "speedup_solves_per_s": round(rb["solves_per_s"] / seq["solves_per_s"], 2)
            if seq["solves_per_s"] else None}


def run_serving(args):
    """--workload serving: the request stream (serving_measure), reduced from
    the full stream (2000 requests, nr up to 1024) by --requests, --nr-lo,
    --nr-hi.  The server stores FP32 by default, so both arms reach the
    steady state at the same Nu accuracy: the criterion |dNu| < 1e-6 lies
    below the rounding noise of 16-bit storage (--serve-storage fp16 runs
    most requests to the step cap)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    m = serving_measure(args.requests, args.nr_lo, args.nr_hi, args.max_steps, args.serve_storage,
                        args.serve_node_budget)
    line = {"metric": METRIC, "value": m["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.serve_storage], "data": "synthetic",
            "config": {"workload": "Poisson stream of axisymmetric solve requests (60 % annulus convection, "
                                   "40 % swirling cylinder), continuous batching", **m["config"]},
            **{k: v for k, v in m.items() if k not in ("solves_per_s", "config")}}
    print(json.dumps(line), flush=True)
    return 0


def batch_measure(instances, lo, hi, storage, steps, warmup, graph_steps, oracle_instances, repeats=1,
                  clocks=None, kind="annuli"):
    """Uneven lattices advanced together by the batched step, replayed from
    CUDA graphs, the launch autotuned per batch: median aggregate MLUPS over
    `repeats` timed regions of `steps` steps, the HBM roofline, and the Nu of
    the smallest instances against the oracle after the same steps.  kind
    "annuli": annulus-convection lattices, nr, nz ~ U{lo..hi}, seeds
    0..instances-1; "requests": the lattices of the serving stream's first
    `instances` requests with nr ~ U{lo..hi} (60 % annuli, 40 % swirling
    cylinders, nz = nr U{1,2})."""
    import numpy as np
    import torch
    import oracle
    from paper_1806_10241_gb300 import autotune
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    if kind == "requests":
        cases = [r.case for r in W.serving_requests(count=instances, rate=50.0, seed=0, nr_lo=lo, nr_hi=hi)]
        desc = (f"{len(cases)} lattices of the serving stream (seed 0): nr ~ U{{{lo}..{hi}}}, nz = nr U{{1,2}}, "
                "60 % annulus convection, 40 % swirling cylinder")
    else:
        cases = W.batched_instances(instances, lo=lo, hi=hi)
        desc = (f"{len(cases)} annulus-convection lattices, nr, nz ~ U{{{lo}..{hi}}}, "
                "R_o/R_i ~ U[1.5,3], Ra log-U[1e3,1e5], inner swirl ~ U[0,0.05], seeds 0..")
    stream = torch.cuda.Stream()
    solvers = []
    for cs in cases:
        s = Solver(cs.params, storage=storage, stream=stream)
        s.init_fields(cs.fields)
        solvers.append(s)
    nodes = sum(cs.nr * cs.nz for cs in cases)
    b = Batch(solvers, stream=stream, graph_steps=graph_steps)
    launch = autotune.tune_batch(b, graph_steps=graph_steps)
    b.step(warmup)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        time.sleep(0.6)
    t0 = time.time()
    ms = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t1 = time.time()
    if clocks is not None:
        clocks.stop()
    med = sorted(ms)[len(ms) // 2]
    peaks, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[storage]
    achieved = bpn * nodes * steps / (med * 1e-3) / 1e9
    order = sorted(range(len(cases)), key=lambda m: cases[m].nr * cases[m].nz)
    pick = [m for m in order if cases[m].nr <= 64 and cases[m].nz <= 64] or order[:oracle_instances]
    nu = []
    for m in pick[:oracle_instances]:
        cs = cases[m]
        o = oracle.Oracle(cs.params)
        o.init_fields(cs.fields)
        o.step(solvers[m].step_count)
        dn, do = solvers[m].diag(), o.diag()
        nu.append({"instance": m, "nr": cs.nr, "nz": cs.nz, "steps": solvers[m].step_count,
                   "nu_gpu": dn["nu_avg"], "nu_oracle": do["nu_avg"],
                   "rel_err": abs(dn["nu_avg"] - do["nu_avg"]) / abs(do["nu_avg"])})
    b.close()
    del solvers
    torch.cuda.empty_cache()
    return {"value": round(nodes * steps / (med * 1e3), 1), "unit": "MLUPS", "steps": steps, "warmup": warmup,
            "repeats": repeats, "ms_per_step": round(med / steps, 5),
            "mlups_range": [round(nodes * steps / (max(ms) * 1e3), 1), round(nodes * steps / (min(ms) * 1e3), 1)],
            "config": {"workload": desc,
                       "nodes": nodes, "storage": storage,
                       "launch": {"seg_rows": launch[0], "warps_per_block": launch[1], "row_fetch": launch[2],
                                  "graph_steps": graph_steps,
                                  "segment_plan_waves": launch[3]},
                       "l2": ("inputs larger than L2 (working set %.0f MB)" % (bpn * nodes / 1e6)
                              if bpn * nodes > L2_BYTES else
                              "working set %.0f MB fits in the L2: an L2-resident rate" % (bpn * nodes / 1e6))},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": round(achieved / float(peaks["hbm_gbs"]), 4), "traffic": None,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_node": bpn,
                         "kernel": "k_batch3 (batched fused step)"},
            "gpu_launches": steps * repeats, "clocks": clocks.summary(t0, t1) if clocks is not None else None,
            "nu_vs_oracle": nu, "dtype": DTYPE[storage]}


def run_batch(args):
    """--workload batch: 256 uneven annulus-convection lattices (batch_measure;
    --instances, --batch-lo, --batch-hi change the count and the size range)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    m = batch_measure(args.instances, args.batch_lo, args.batch_hi, args.batch_storage, args.steps, args.warmup,
                      args.graph_steps, args.oracle_instances, repeats=max(1, args.repeats),
                      clocks=ClockSampler(0), kind=args.batch_set)
    line = {"metric": METRIC, "value": m["value"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": m["dtype"], "data": "synthetic",
            **{k: v for k, v in m.items() if k not in ("value", "unit", "steps", "warmup", "ms_per_step", "dtype")}}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """--workload precision: the 16-bit storage forms of the benchmark
    cylinder.  MLUPS of each storage at 1024 x 2048, the errors of FP32, FP16
    and BF16 against the GPU FP64 path at full size, and against the FP64
    oracle on a 256 x 512 copy (Re = 1000 on R)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.solver import Solver
    torch.cuda.set_device(0)

    def rel_l2(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    def errors(f, d, fr, dr):
        e = {fld: rel_l2(f[q], fr[q]) for q, fld in ((1, "u_z"), (2, "u_r"), (3, "u_theta"), (4, "T"))}
        e["nu_avg"] = abs(d["nu_avg"] - dr["nu_avg"]) / abs(dr["nu_avg"])
        return {k: float("%.3g" % v) for k, v in e.items()}

    steps = args.prec_steps
    case = W.config_cylinder(args.nr, args.nz)
    nodes = case.nr * case.nz
    res, mlups = {}, {}
    for storage in ("fp64", "fp32", "fp16", "bf16"):
        g = Solver(case.params, storage=storage)
        g.init_fields(case.fields)
        g.step(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.step(steps - 3)
        e1.record(g.stream)
        e1.synchronize()
        mlups[storage] = round(nodes * (steps - 3) / (e0.elapsed_time(e1) * 1e3), 1)
        res[storage] = (g.fields(), g.diag())
        del g
        torch.cuda.empty_cache()
    full = {s: errors(*res[s], *res["fp64"]) for s in ("fp32", "fp16", "bf16")}
    small = W.swirling_cylinder(nr=256, nz=512, Re=1000.0, Ra=1e5, Pr=0.7, u_lid=0.05, amp=1e-6, seed=0)
    o = oracle.Oracle(small.params)
    o.init_fields(small.fields)
    o.step(args.prec_oracle_steps)
    ref = (o.fields(), o.diag())
    copy = {}
    for storage in ("fp32", "fp16", "bf16"):
        g = Solver(small.params, storage=storage)
        g.init_fields(small.fields)
        g.step(args.prec_oracle_steps)
        copy[storage] = errors(g.fields(), g.diag(), *ref)
    line = {"metric": METRIC, "value": mlups["fp16"], "unit": "MLUPS", "n_gpus": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE["fp16"], "data": "synthetic",
            "config": {"workload": workload_desc(case.nr, case.nz, "fp16/bf16/fp32/fp64"), "steps": steps},
            "mlups": mlups,
            "speedup_vs_fp32": {s: round(mlups[s] / mlups["fp32"], 3) for s in ("fp16", "bf16")},
            "rel_err_vs_gpu_fp64_full_size": full,
            "rel_err_vs_oracle_256x512": {"steps": args.prec_oracle_steps, **copy},
            "nu_avg": {s: res[s][1]["nu_avg"] for s in res}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, K steps after W
    warm-up steps, each step a bounded slab of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1806_10241_gb300 import workloads as W
    oracle.build()
    nr, nz = args.nr, args.nz
    # size the slab so the whole run ends in about two minutes
    probe = W.config_cylinder(nr, 16)
    o = oracle.Oracle(probe.params)
    o.init_fields(probe.fields)
    t = time.perf_counter()
    o.step(2)
    rate = 2 * nr * 16 / max(time.perf_counter() - t, 1e-6)  # node updates / s
    total = args.steps + args.warmup
    rows = int(max(4, min(nz, 120.0 * rate / (total * nr))))
    c = W.config_cylinder(nr, rows)
    o = oracle.Oracle(c.params)
    o.init_fields(c.fields)
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    v = nr * rows * args.steps / dt / 1e6
    threads = oracle.get_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(nr, nz, args.storage), "nr": nr, "nz": nz,
                       "storage": args.storage, "parallelism": "replicas",
                       "oracle": f"FP64, a {nr}x{rows} slab of the lattice per step (same per-node work)"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} steps of a {nr}x{rows} slab after {args.warmup} "
                                       f"warm-up steps, {threads} OpenMP threads"},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def storage_forms(case, steps, warmup, repeats, sm_mhz=None):
    """The benchmark lattice in FP32, FP16 and BF16 storage, each from the
    same initial state: `warmup` steps, then `repeats` timed regions of
    `steps` steps (median); Nu of the 16-bit forms against the FP32 run after
    the same number of steps."""
    import torch
    from paper_1806_10241_gb300.solver import Solver
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    nodes = case.nr * case.nz
    out = {}
    for storage in ("fp32", "fp16", "bf16"):
        g = Solver(case.params, storage=storage)
        g.init_fields(case.fields)
        g.step(warmup)
        ms = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(g.stream)
            g.step(steps)
            e1.record(g.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = sorted(ms)[len(ms) // 2]
        d = g.diag()
        bpn = BYTES_PER_NODE[storage]
        out[storage] = {"value": round(nodes * steps / (med * 1e3), 1), "unit": "MLUPS",
                        "ms_per_step": round(med / steps, 5), "launch": list(g.get_launch()),
                        "roofline_frac": round(bpn * nodes / (med / steps * 1e-3) / 1e9 / peak, 4),
                        "algorithmic_bytes_per_node": bpn, "nu_avg": d["nu_avg"],
                        "steps_total": warmup + steps * repeats, "status": d["status"]}
        kname = kernel_name(storage, g.get_launch()[2])
        iss = issue_roofline(f"{kname}_{storage}_{case.nr}x{case.nz}", med / steps, sm_mhz)
        if iss is not None:
            out[storage]["issue"] = iss
        del g
        torch.cuda.empty_cache()
    for storage in ("fp16", "bf16"):
        e = out[storage]
        e["speedup_vs_fp32"] = round(e["value"] / out["fp32"]["value"], 3)
        e["nu_rel_diff_vs_fp32"] = abs(e["nu_avg"] - out["fp32"]["nu_avg"]) / abs(out["fp32"]["nu_avg"])
    return out


def extras(case, args, sm_mhz=None):
    """Sub-results measured in the same run, a few seconds each: the 16-bit
    storage forms of the benchmark lattice, the 256-lattice batch and a short
    serving stream."""
    res = {}
    forms = storage_forms(case, steps=500, warmup=50, repeats=10, sm_mhz=sm_mhz)
    res["fp16"] = forms["fp16"]
    res["bf16"] = forms["bf16"]
    res["fp16"]["fp32_same_schedule"] = {k: forms["fp32"][k] for k in ("value", "ms_per_step", "nu_avg")}
    res["bf16"]["fp32_same_schedule"] = res["fp16"]["fp32_same_schedule"]
    b = batch_measure(256, 32, 512, "fp16", steps=100, warmup=20, graph_steps=50, oracle_instances=3, repeats=5)
    res["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "mlups_range", "config", "nu_vs_oracle")}
    res["batch"]["roofline_frac"] = b["roofline"]["frac"]
    sv = serving_measure(args.serve_requests, 64, 96, args.serve_max_steps, "fp32")
    res["serving"] = {"solves_per_s": sv["solves_per_s"], "p50_latency_s": sv["p50_latency_s"],
                      "p99_latency_s": sv["p99_latency_s"],
                      "sequential_fp32": {k: sv["sequential_fp32"][k] for k in
                                          ("solves_per_s", "p50_latency_s", "p99_latency_s", "converged",
                                           "capped", "diverged")},
                      "batched": {k: sv["batched"][k] for k in ("converged", "capped", "diverged", "rounds",
                                                                "max_concurrent")},
                      "speedup_solves_per_s": sv["speedup_solves_per_s"],
                      "nu_rel_diff_vs_sequential_fp32": sv["nu_rel_diff_vs_sequential_fp32"],
                      "config": sv["config"]}
    return res


# ---- the GPU arm ----------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"])
    ap.add_argument("--nr", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 16-bit, batch and serving sub-results of the default line")
    ap.add_argument("--repeats", type=int, default=0,
                    help="timed regions of K steps (0: automatic, 5..20); the line reports the median")
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=16)
    ap.add_argument("--serve-node-budget", dest="serve_node_budget", type=int, default=0,
                    help="--workload serving: at most this many nodes stepped together (0: HBM admission only)")
    ap.add_argument("--serve-max-steps", dest="serve_max_steps", type=int, default=50_000)
    ap.add_argument("--workload", default="cylinder", choices=["cylinder", "serving", "precision", "batch"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--batch-storage", dest="batch_storage", default="fp16", choices=["fp16", "bf16", "fp32"])
    ap.add_argument("--batch-set", dest="batch_set", default="annuli", choices=["annuli", "requests"],
                    help="batch of uneven annuli, or the lattices of the serving stream's first requests")
    ap.add_argument("--batch-lo", dest="batch_lo", type=int, default=32)
    ap.add_argument("--batch-hi", dest="batch_hi", type=int, default=512)
    ap.add_argument("--graph-steps", dest="graph_steps", type=int, default=50)
    ap.add_argument("--oracle-instances", dest="oracle_instances", type=int, default=3)
    ap.add_argument("--prec-steps", dest="prec_steps", type=int, default=2000)
    ap.add_argument("--prec-oracle-steps", dest="prec_oracle_steps", type=int, default=1500)
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--nr-lo", dest="nr_lo", type=int, default=64)
    ap.add_argument("--nr-hi", dest="nr_hi", type=int, default=128)
    ap.add_argument("--max-steps", dest="max_steps", type=int, default=200_000)
    ap.add_argument("--serve-storage", dest="serve_storage", default="fp32", choices=["fp16", "bf16", "fp32"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "batch":
        return run_batch(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.solver import Solver

    case = W.config_cylinder(args.nr, args.nz)
    nodes = case.nr * case.nz
    g = Solver(case.params, storage=args.storage, device=dev)
    stream = g.stream
    g.init_fields(case.fields)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    g.step(args.warmup)
    barrier()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.6)

    # device-timed regions: K steps each, one fused kernel per step, inputs
    # resident; the same number of regions on every rank, each bracketed by a
    # barrier and a synchronisation, its time the max over the ranks
    def region():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.step(args.steps)
            e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    t0 = time.time()
    ms_all = [region()]
    repeats = args.repeats
    if repeats <= 0:  # automatic: about a second of timed work, 5..20 regions
        repeats = int(min(20, max(5, 1000.0 / max(ms_all[0], 1e-3))))
        repeats = int(max_over_ranks(repeats, dist, dev))  # every rank runs the same count
    for _ in range(repeats - 1):
        ms_all.append(region())
    t1 = time.time()
    clocks.stop()
    ms_sorted = sorted(ms_all)
    ms = ms_sorted[len(ms_sorted) // 2]  # median region
    ms_per_step = ms / args.steps
    value = job_mlups(world, nodes, args.steps, ms)  # MLUPS, whole job
    d = g.diag()

    # end to end through the C ABI with host buffers: a 2000-step solve that
    # uploads the initial fields from pinned memory, steps and downloads the
    # fields
    host_in = torch.from_numpy(np.ascontiguousarray(case.fields)).pin_memory()
    host_out = torch.empty((5, case.nz, case.nr), dtype=torch.float64).pin_memory()
    ge = Solver(case.params, storage=args.storage, device=dev)
    e_steps = 2000
    e_times = []
    for _ in range(3):  # three solves, the median reported (host-side timing varies)
        barrier()
        t = time.perf_counter()
        ge.init_fields(host_in.numpy())
        ge.step(e_steps)
        ge.fields(out=host_out.numpy())
        barrier()
        e_times.append(max_over_ranks(time.perf_counter() - t, dist, dev))
    e2e_s = sorted(e_times)[1]
    e2e = {"value": round(world * nodes * e_steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(host_in.numel() * 8 / e_steps),
           "d2h_bytes_per_step": int(host_out.numel() * 8 / e_steps),
           "steps": e_steps, "solves": len(e_times), "statistic": "median solve",
           "what": "one solve: lb_init_fields (pinned host fields) + 2000 lb_step + lb_get_fields to host"}
    del ge

    peaks, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[args.storage]
    achieved = bpn * nodes / (ms_per_step * 1e-3) / 1e9  # GB/s of one launch
    peak = float(peaks["hbm_gbs"])
    seg, wpb, fetch = g.get_launch()
    kname = kernel_name(args.storage, fetch)
    key = f"{kname}_{args.storage}_{case.nr}x{case.nz}"
    traffic = counters_for(key)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "frac_of_nominal_7900_GBs": round(achieved / 7900.0, 4),
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_node": bpn,
                "kernel": f"{kname} (fused stream + sources + collisions + boundaries, one launch per step)"}

    clk = clocks.summary(t0, t1)
    iss = issue_roofline(key, ms_per_step, clk.get("sm_mhz"))
    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.storage], "data": "synthetic",
            "config": {"workload": workload_desc(case.nr, case.nz, args.storage), "nr": case.nr,
                       "nz": case.nz, "storage": args.storage, "parallelism": "replicas",
                       "launch": {"seg_rows": seg, "warps_per_block": wpb, "row_fetch": fetch},
                       "l2": "inputs larger than L2 (working set %.0f MB)" % (2 * 19 * nodes *
                                                                          bpn / 38 / 1e6)},
            "repeats": {"regions": len(ms_all), "statistic": "median region of K steps",
                        "mlups_min": round(job_mlups(world, nodes, args.steps, ms_sorted[-1]), 1),
                        "mlups_max": round(job_mlups(world, nodes, args.steps, ms_sorted[0]), 1)},
            "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps * len(ms_all),
            "clocks": clk,
            "diag": {"nu_avg": d["nu_avg"], "mass": d["mass"], "status": d["status"]}}
    if iss is not None:
        line["issue_roofline"] = iss  # the same kernel against the schedulers' issue ceiling, for context
    del g
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(extras(case, args, clk.get("sm_mhz")))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_mlups(case.nr, case.nz, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
