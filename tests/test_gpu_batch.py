"""Batched step: each lattice's result is the same alone and in a batch of
uneven lattices (bitwise: the per-lattice arithmetic and rounding bits are
identical), and matches the FP64 oracle like a single lattice does."""
import numpy as np
import pytest

import oracle
from paper_1806_10241_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()
    oracle.build()


def _cases():
    cs = W.batched_instances(count=6, lo=20, hi=150)
    cs.append(W.swirling_cylinder(nr=70, nz=45, Re=200.0, Ra=1e4, amp=1e-3, seed=9))
    cs.append(W.taylor_couette(R_o=40, beta=0.5))
    return cs


@pytest.mark.parametrize("row_fetch", [1, 2, 3])
@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_batch_equals_individual_runs(storage, row_fetch):
    """The batched step and the single-lattice step with each row fetch give
    the same bits (16-bit storage included: the rounding draws depend only on
    the node, the plane and the step)."""
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    cases = _cases()
    alone = []
    for c in cases:
        s = Solver(c.params, storage=storage, stream=stream)
        s.set_launch(0, 0, row_fetch)
        s.init_fields(c.fields)
        s.step(56)
        alone.append(s.get_dist())
    mixed = []
    for c in cases:
        s = Solver(c.params, storage=storage, stream=stream)
        s.init_fields(c.fields)
        mixed.append(s)
    b = Batch(mixed, stream=stream, graph_steps=8)  # TMA ring read in place, one warp per item
    b.step(5)
    b.set_launch(seg_rows=5, warps_per_block=4, graph_steps=4, row_fetch=1)  # plain loads, persistent grid
    b.step(16)  # 4 graph replays of 4 launches
    b.set_launch(seg_rows=3, warps_per_block=2, graph_steps=4, row_fetch=3)
    b.step(11)  # 2 graph replays, then 3 launches outside the graph
    b.step(5)  # 1 replay, 1 launch
    # per-lattice segments (0: the common value; 31 = the whole height of lattice 3)
    b.set_segments([1, 7, 2, 31, 0, 3, 11, 3])
    b.step(6)
    b.set_segments(None)
    b.step(1)
    if storage == "fp32":  # three ring stages
        b.set_launch(seg_rows=4, warps_per_block=2, graph_steps=4, row_fetch=4)
        b.step(5)
    else:
        b.step(5)
    # one persistent launch per call, items waiting on their neighbours' progress
    b.set_launch(seg_rows=3, warps_per_block=2, graph_steps=0, row_fetch=5)
    resident, items = b.occupancy()
    assert items <= resident
    b.step(6)
    b.step(1)
    torch.cuda.synchronize()
    for c, a, s in zip(cases, alone, mixed):
        assert s.step_count == 56
        assert np.array_equal(s.get_dist(), a), c.name
    b.close()


# every boundary family of the single-lattice parity tests, at widths of one
# and two 64-column windows and heights that split into uneven segments
FAMILY_SHAPES = {"annulus_walls": (65, 23), "cylinder_axis": (33, 17), "periodic_annulus": (97, 12),
                 "periodic_cylinder": (128, 9), "planar_box": (7, 9), "rotating_cylinder": (61, 13),
                 "sliding_annulus": (70, 8), "czochralski": (40, 31), "free_ends_annulus": (100, 20)}


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_batch_of_every_boundary_family_equals_individual_runs(storage):
    """Lattices of every boundary family (walls sliding, porous and rotating,
    the axis, periodic ends, the planar form, rigid rotation, the Czochralski
    split top with a free surface and the surface ramp, free surfaces at both
    ends) from seeded random states, batched together through each launch
    path, give the bits of the single-lattice step."""
    from test_gpu_parity import BUILDERS, random_state
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    params = [BUILDERS[name](*shape) for name, shape in FAMILY_SHAPES.items()]
    states = [random_state(p, seed) for seed, p in enumerate(params)]
    alone = []
    for p, st in zip(params, states):
        s = Solver(p, storage=storage, stream=stream)
        s.set_dist(st)
        s.step(40)
        alone.append(s.get_dist())
    sols = []
    for p, st in zip(params, states):
        s = Solver(p, storage=storage, stream=stream)
        s.set_dist(st)
        sols.append(s)
    b = Batch(sols, stream=stream, graph_steps=4)
    b.step(9)  # TMA ring, graphs of 4 launches and one launch outside
    b.set_launch(seg_rows=5, warps_per_block=2, graph_steps=0, row_fetch=1)
    b.step(7)  # plain loads
    b.set_segments([3, 0, 2, 9, 1, 13, 4, 6, 5])
    b.set_launch(seg_rows=4, warps_per_block=1, graph_steps=3, row_fetch=4 if storage == "fp32" else 3)
    b.step(8)
    b.set_segments(None)
    b.set_launch(seg_rows=3, warps_per_block=2, graph_steps=0, row_fetch=5)
    resident, items = b.occupancy()
    assert items <= resident
    b.step(16)  # one persistent launch
    torch.cuda.synchronize()
    for name, a, s in zip(FAMILY_SHAPES, alone, sols):
        assert s.step_count == 40
        assert np.array_equal(s.get_dist(), a), name
    # the batched diagnostics (one grid for all lattices) are those of each lattice
    together = b.diag()
    for name, t, s in zip(FAMILY_SHAPES, together, sols):
        assert t["status"] == 0, name
        assert t == s.diag(), name
    b.close()


def test_batch_matches_oracle_fp32():
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    cases = _cases()[:4]
    sols = []
    for c in cases:
        s = Solver(c.params, storage="fp32")
        s.init_fields(c.fields)
        sols.append(s)
    b = Batch(sols, stream=torch.cuda.Stream(), graph_steps=10)
    b.step(300)
    torch.cuda.synchronize()
    for c, s in zip(cases, sols):
        o = oracle.Oracle(c.params)
        o.init_fields(c.fields)
        o.step(300)
        got, want = s.fields(), o.fields()
        for q in (1, 2, 4):
            n = np.linalg.norm(want[q])
            if n > 0:
                assert np.linalg.norm(got[q] - want[q]) / n < 1e-5, (c.name, q)
        d = s.diag()
        assert d["status"] == 0 and d["step"] == 300


def test_batch_diagnostics_equal_per_lattice_diagnostics():
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    sols = []
    for c in _cases():
        s = Solver(c.params, storage="fp16", stream=stream)
        s.init_fields(c.fields)
        sols.append(s)
    b = Batch(sols, stream=stream, graph_steps=5)
    b.step(25)
    together = b.diag()
    alone = [s.diag() for s in sols]
    for t, a in zip(together, alone):
        assert t == a
    b.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_of_many_lattices_equals_individual_runs(storage):
    """70 small lattices: the instance lookup takes two rounds of its ballot
    search (more than 32 instances), and a step count that is not a multiple
    of the graph length mixes graph replays with single launches.  Every
    lattice ends bitwise as it does alone."""
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    cases = W.batched_instances(count=70, lo=8, hi=70)
    alone = []
    for c in cases:
        s = Solver(c.params, storage=storage, stream=stream)
        s.init_fields(c.fields)
        s.step(23)
        alone.append(s.get_dist())
    mixed = []
    for c in cases:
        s = Solver(c.params, storage=storage, stream=stream)
        s.init_fields(c.fields)
        mixed.append(s)
    b = Batch(mixed, stream=stream, graph_steps=10)
    b.step(23)
    torch.cuda.synchronize()
    for c, a, s in zip(cases, alone, mixed):
        assert s.step_count == 23
        assert np.array_equal(s.get_dist(), a), c.name
    b.close()


def test_batch_diagnostics_follow_a_changed_launch():
    """A lattice whose launch settings change between two calls gets the
    diagnostics grid of its new settings: still bitwise its own diagnostics."""
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    stream = torch.cuda.Stream()
    sols = []
    for c in _cases()[:5]:
        s = Solver(c.params, storage="fp32", stream=stream)
        s.init_fields(c.fields)
        sols.append(s)
    b = Batch(sols, stream=stream, graph_steps=5)
    b.step(12)
    assert b.diag() == [s.diag() for s in sols]
    sols[2].set_launch(48, 2, 0)  # 48-row segments: another diagnostics grid
    b.step(3)
    assert b.diag() == [s.diag() for s in sols]
    b.close()


def test_batch_orders_work_queued_on_the_lattices_own_streams():
    """Each lattice on a stream of its own, the batch on another: work queued
    on a lattice's stream (initial fields, a state upload) runs before the
    batch's next step, and the batch's steps before the lattice's next
    download, without any synchronisation by the caller."""
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    cases = _cases()[:5]
    ref = []
    for c in cases:
        s = Solver(c.params, storage="fp32")
        s.init_fields(c.fields)
        s.step(30)
        if c is cases[2]:
            s.set_dist(s.get_dist() * 1.0001)
        s.step(20)
        ref.append(s.get_dist())
        s.close()
    sols = []
    for c in cases:
        s = Solver(c.params, storage="fp32", stream=torch.cuda.Stream())
        s.init_fields(c.fields)  # queued on the lattice's stream
        sols.append(s)
    b = Batch(sols, stream=torch.cuda.Stream(), graph_steps=10)
    b.step(30)
    mid = sols[2].get_dist()  # on the lattice's stream, after the batch's steps
    sols[2].set_dist(mid * 1.0001)
    b.step(20)
    for c, s, want in zip(cases, sols, ref):
        assert np.array_equal(s.get_dist(), want), c.name
    b.close()


def test_segment_plan_rejects_out_of_range_values():
    from paper_1806_10241_gb300._abi import LBError
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    cases = _cases()[:3]
    sols = []
    for c in cases:
        s = Solver(c.params, storage="fp32")
        s.init_fields(c.fields)
        sols.append(s)
    b = Batch(sols, stream=torch.cuda.Stream())
    with pytest.raises(LBError):
        b.set_segments([1, -1, 2])
    with pytest.raises(LBError):
        b.set_segments([1, cases[1].nz + 1, 2])
    b.set_launch(row_fetch=4)
    r4, _ = b.occupancy()
    b.set_launch(row_fetch=3)
    resident, items = b.occupancy()
    assert resident >= 152 and items > 0
    assert r4 > resident  # three stages: more warps resident
    b.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_persistent_batch_equals_launch_per_step(storage):
    """Row fetch 5 (one cooperative launch for all the steps of a call) gives
    the bits of one launch per step, over a long call on uneven lattices with
    a periodic one among them (z-segments that wrap)."""
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    cases = _cases()
    runs = []
    for fetch in (3, 5):
        stream = torch.cuda.Stream()
        sols = []
        for c in cases:
            s = Solver(c.params, storage=storage, stream=stream)
            s.init_fields(c.fields)
            sols.append(s)
        b = Batch(sols, stream=stream, seg_rows=5, warps_per_block=2, graph_steps=0, row_fetch=fetch)
        b.step(150)
        torch.cuda.synchronize()
        assert all(d["status"] == 0 for d in b.diag())
        runs.append([s.get_dist() for s in sols])
        b.close()
    for c, a, p in zip(cases, runs[0], runs[1]):
        assert np.array_equal(a, p), c.name


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_persistent_batch_over_every_boundary_family_for_1000_steps(storage):
    """Row fetch 5 over lattices of every boundary family, 1000 steps in
    calls of uneven length (each a persistent launch whose items wait on
    their neighbours' progress), against one launch per step: the same bits."""
    from test_gpu_parity import BUILDERS, random_state
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    params = [BUILDERS[name](*shape) for name, shape in FAMILY_SHAPES.items()]
    states = [random_state(p, seed) for seed, p in enumerate(params)]
    runs = []
    for fetch, seg, graph, call in ((3, 4, 10, 500), (5, 3, 0, 97)):
        stream = torch.cuda.Stream()
        sols = []
        for p, st in zip(params, states):
            s = Solver(p, storage=storage, stream=stream)
            s.set_dist(st)
            sols.append(s)
        b = Batch(sols, stream=stream, seg_rows=seg, warps_per_block=2, graph_steps=graph, row_fetch=fetch)
        left = 1000
        while left > 0:
            b.step(min(left, call))
            left -= call
        torch.cuda.synchronize()
        assert all(d["status"] != _abi.LB_ERR_TIMEOUT for d in b.diag())  # no wait ran out
        runs.append([s.get_dist() for s in sols])
        b.close()
    for name, a, p in zip(FAMILY_SHAPES, runs[0], runs[1]):
        assert np.array_equal(a, p), name


def test_persistent_batch_rejects_more_items_than_resident_warps():
    from paper_1806_10241_gb300._abi import LBError
    from paper_1806_10241_gb300.batch import Batch
    from paper_1806_10241_gb300.solver import Solver
    c = W.swirling_cylinder(nr=1024, nz=2048, amp=0.0)
    s = Solver(c.params, storage="fp32")
    b = Batch([s], stream=torch.cuda.Stream(), seg_rows=4, row_fetch=5)
    resident, items = b.occupancy()
    assert items > resident
    with pytest.raises(LBError):
        b.step(1)
    b.close()
