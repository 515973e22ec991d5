"""Serving loop: continuous batching with admission by a device-memory
budget.  Every request finishes, requests overlap on the device, and each
result is bitwise the one of the same request run alone for the same steps."""
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


def _stream(n=7):
    out = []
    for i in range(n):
        nr = 16 + 6 * i
        c = W.annulus_convection(nr=nr, nz=nr + 8 * (i % 3), Ra=10 ** (3 + (i % 3) * 0.5), amp=1e-4, seed=i,
                                 swirl_inner=0.01 * (i % 2))
        c.name = f"r{i}"
        # half of the stream at once (so that requests share the device however
        # fast each one finishes), the rest arriving while those run
        out.append(W.Request(i, 0.0 if i % 2 == 0 else 0.003 * i, c))
    return out


def _alone(req, steps, storage, rounds):
    from paper_1806_10241_gb300.solver import Solver
    s = Solver(req.case.params, storage=storage)
    s.init_fields(req.case.fields)
    for _ in range(steps // rounds):
        s.step(rounds)
    return s.get_dist()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_server_results_equal_solo_runs(storage):
    from paper_1806_10241_gb300.serving import Server
    reqs = _stream()
    srv = Server(storage=storage, steps_per_round=100, check_every=200, window=400, tol=1e-7,
                 max_steps=2000, keep_results=True, graph_steps=5)
    rep = srv.run(reqs)
    summ = rep.summary()
    assert summ["completed"] == len(reqs)
    assert srv.max_concurrent >= 2  # requests overlapped on the device
    for r in rep.records:
        assert r.status in ("converged", "capped"), (r.name, r.status)
        assert r.steps > 0 and r.latency > 0
        want = _alone(reqs[r.rid], r.steps, storage, 100)
        assert np.array_equal(srv.results[r.rid], want), r.name


def test_admission_respects_the_memory_budget():
    from paper_1806_10241_gb300.serving import Server
    from paper_1806_10241_gb300.solver import required_bytes
    reqs = [W.Request(r.rid, 0.0, r.case) for r in _stream(6)]  # a burst: all at once
    biggest = max(required_bytes(r.case.params, "fp16") for r in reqs)
    srv = Server(storage="fp16", steps_per_round=100, check_every=200, window=400, tol=1e-7, max_steps=800,
                 hbm_budget=2 * biggest + 1)
    rep = srv.run(reqs)
    assert rep.summary()["completed"] == len(reqs)
    assert srv.max_concurrent <= 2
    # later requests waited for memory
    waited = [r for r in rep.records if r.admitted - r.arrival > 1e-3]
    assert waited


def test_sequential_baseline_runs():
    from paper_1806_10241_gb300.serving import Server
    reqs = _stream(3)
    srv = Server(storage="fp16", steps_per_round=100, check_every=200, window=400, tol=1e-7, max_steps=600)
    rep = srv.run_sequential(reqs, storage="fp32")
    s = rep.summary()
    assert s["completed"] == 3 and s["p99_latency_s"] >= s["p50_latency_s"]


def test_oversize_request_is_rejected_and_the_rest_complete():
    from paper_1806_10241_gb300.serving import Server
    from paper_1806_10241_gb300.solver import required_bytes
    reqs = [W.Request(r.rid, 0.0, r.case) for r in _stream(3)]
    biggest = max(required_bytes(r.case.params, "fp16") for r in reqs)
    huge = W.annulus_convection(nr=2048, nz=4096, Ra=1e4)
    reqs.append(W.Request(99, 0.0, huge))
    assert required_bytes(huge.params, "fp16") > 2 * biggest + 1
    srv = Server(storage="fp16", steps_per_round=100, check_every=200, window=400, tol=1e-7, max_steps=400,
                 hbm_budget=2 * biggest + 1)
    rep = srv.run(reqs)
    st = {r.rid: r.status for r in rep.records}
    assert st[99] == "rejected"
    assert all(st[r.rid] in ("converged", "capped") for r in reqs[:3])
    s = rep.summary()
    assert s["rejected"] == 1 and s["completed"] == 4


def test_cancelled_requests_leave_the_batch():
    from paper_1806_10241_gb300.serving import Server
    reqs = [W.Request(r.rid, 0.0, r.case) for r in _stream(4)]
    srv = Server(storage="fp16", steps_per_round=100, check_every=200, window=400, tol=1e-9, max_steps=1000,
                 max_active=2)

    def on_round(server, now):
        server.cancel(0)  # active from the first round
        server.cancel(3)  # still waiting for a slot

    rep = srv.run(reqs, on_round=on_round)
    st = {r.rid: r for r in rep.records}
    assert st[0].status == "cancelled" and st[0].steps == 100
    assert st[3].status == "cancelled" and st[3].admitted < 0
    assert st[1].status in ("converged", "capped") and st[2].status in ("converged", "capped")
    assert rep.summary()["cancelled"] == 2


def test_diverged_lattice_is_reported_and_retired():
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300.serving import Server
    from paper_1806_10241_gb300.solver import Solver
    bad = W.annulus_convection(nr=24, nz=24, Ra=1e4, seed=1)
    bad.fields = bad.fields.copy()
    bad.fields[4, 5, 7] = np.nan  # a NaN temperature in the request's initial state
    s = Solver(bad.params, storage="fp32")
    s.init_fields(bad.fields)
    s.step(5)
    assert s.diag()["status"] == _abi.LB_ERR_DIVERGED
    reqs = [W.Request(0, 0.0, bad)] + [W.Request(r.rid + 1, 0.0, r.case) for r in _stream(2)]
    srv = Server(storage="fp16", steps_per_round=100, check_every=200, window=400, tol=1e-7, max_steps=400)
    rep = srv.run(reqs)
    st = {r.rid: r.status for r in rep.records}
    assert st[0] == "diverged"
    assert st[1] in ("converged", "capped") and st[2] in ("converged", "capped")


def test_autotuned_server_gives_the_same_results_as_solo_runs():
    """Autotuning rebuilds of the batch changes launches and adds real steps;
    each request's result is still bitwise the one of its solo run for the
    same number of steps."""
    from paper_1806_10241_gb300 import autotune
    from paper_1806_10241_gb300.serving import Server
    from paper_1806_10241_gb300.solver import Solver
    reqs = _stream(4)
    srv = Server(storage="fp32", steps_per_round=100, check_every=200, window=400, tol=1e-9, max_steps=600,
                 keep_results=True, autotune=True)
    rep = srv.run(reqs)
    for r in rep.records:
        req = reqs[r.rid]
        s = Solver(req.case.params, storage="fp32")
        s.init_fields(req.case.fields)
        s.step(r.steps)
        assert np.array_equal(srv.results[r.rid], s.get_dist()), r.rid


def test_node_budget_limits_the_lattices_stepped_together():
    """With a node budget the server steps at most that many nodes at once
    (a lone larger request excepted), queues the rest in arrival order, and
    every request still finishes with the result of a solo run."""
    from paper_1806_10241_gb300.serving import Server
    reqs = [W.Request(r.rid, 0.0, r.case) for r in _stream()]  # all waiting at the start
    budget = 2 * max(r.case.nr * r.case.nz for r in reqs)
    srv = Server(storage="fp32", steps_per_round=100, check_every=200, window=400, tol=1e-7,
                 max_steps=1000, keep_results=True, graph_steps=5, node_budget=budget)
    rep = srv.run(reqs)
    assert rep.summary()["completed"] == len(reqs)
    assert 2 <= srv.max_concurrent < len(reqs)
    assert srv.max_nodes <= budget
    admitted = sorted(rep.records, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in admitted] == sorted(r.rid for r in rep.records)  # arrival order
    for r in rep.records:
        assert np.array_equal(srv.results[r.rid], _alone(reqs[r.rid], r.steps, "fp32", 100)), r.name


def test_autotuned_server_stops_every_request_where_a_solo_run_does(tmp_path, monkeypatch):
    """With an empty autotuner cache the server times the launch candidates on
    scratch copies of the active lattices, so the live ones take no extra
    steps: every request is checked at the same steps as in a sequential solo
    run, reaches the same outcome at the same step, and ends in the same bits."""
    from paper_1806_10241_gb300 import autotune
    from paper_1806_10241_gb300.serving import Server
    monkeypatch.setattr(autotune, "_CACHE", str(tmp_path / "autotune.json"))
    reqs = _stream(5)
    kw = dict(steps_per_round=100, check_every=200, window=400, tol=1e-7, max_steps=1400)
    srv = Server(storage="fp32", keep_results=True, autotune=True, **kw)
    rep = srv.run(reqs)
    assert (tmp_path / "autotune.json").exists()  # the candidates were timed
    seq = Server(storage="fp32", **kw).run_sequential(reqs, storage="fp32")
    got = {r.rid: r for r in rep.records}
    for r in seq.records:
        assert (got[r.rid].status, got[r.rid].steps) == (r.status, r.steps), r.rid
        assert got[r.rid].nu == r.nu, r.rid
        want = _alone(reqs[r.rid], r.steps, "fp32", 100)
        assert np.array_equal(srv.results[r.rid], want), r.rid
