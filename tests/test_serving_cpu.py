"""Host logic of the serving loop: the steady-state test and the report."""
import math

from paper_1806_10241_gb300.serving import Record, Report, _steady


def test_steady_state_needs_a_full_window():
    h = [(0, 1.0), (500, 1.0)]
    assert not _steady(h, 1000, 1e-6)  # no sample a full window back yet
    h.append((1000, 1.0 + 5e-7))
    assert _steady(h, 1000, 1e-6)
    h.append((1500, 1.0 + 3e-6))
    assert not _steady(h, 1000, 1e-6)  # compares with step 500
    assert not _steady([(0, 2.0)], 0, 1.0)


def test_report_counts_and_latency_percentiles():
    recs = []
    for i in range(10):
        r = Record(i, f"r{i}", 100, arrival=0.1 * i, admitted=0.1 * i, finished=0.1 * i + 1.0 + 0.1 * i,
                   steps=1000, nu=1.0, status="converged" if i % 2 == 0 else "capped")
        recs.append(r)
    recs.append(Record(10, "big", 10 ** 9, arrival=0.0, finished=0.0, status="rejected"))
    recs.append(Record(11, "gone", 100, arrival=0.5, finished=0.6, status="cancelled"))
    s = Report(recs, makespan=4.0, mode="batched").summary()
    assert s["completed"] == 12 and s["converged"] == 5 and s["capped"] == 5
    assert s["rejected"] == 1 and s["cancelled"] == 1
    assert s["solves_per_s"] == 10 / 4.0  # rejected and cancelled requests are not solves
    lat = sorted(1.0 + 0.1 * i for i in range(10))
    assert math.isclose(s["p50_latency_s"], round((lat[4] + lat[5]) / 2, 3))
    assert s["p99_latency_s"] <= lat[-1] + 1e-9 and s["p99_latency_s"] >= lat[-2]
    assert s["MLUPS"] == round(10 * 1000 * 100 / 4.0 / 1e6, 1)
