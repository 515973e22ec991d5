"""lb_diagnostics_static: diagnostics of a device-resident state without a
context and without scratch memory from the caller.

It serves callers that cannot allocate device memory (a fixed arena handed
out at start-up, or a tool reading checkpoints another component staged in
device memory): they hold only the state, so the entry point keeps its
reduction scratch in the library's own static device array.  Here the
caller's state is a checkpoint blob (lb_get_state) copied into device memory,
and the result must equal lb_diagnostics on the same state, on two calls in
a row.  Collected last (file name) so that a failure here cannot hide the
other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FIELDS = ("nu_i", "nu_o", "nu_avg", "mass", "mass_r", "T_sum", "u_max", "k_eq_i", "k_eq_o")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()


def _static_diag(solver, step):
    """Call the entry point through the C ABI on a device copy of the
    solver's current state."""
    from paper_1806_10241_gb300 import _abi
    L = _abi.load()
    blob = solver.get_state()
    payload = np.frombuffer(blob, dtype=np.uint8)[16:].copy()
    dev = torch.from_numpy(payload).to(solver.device)  # the caller's own memory
    desc = _abi.make_desc(solver.params, solver.storage)
    params = _abi.make_params(solver.params)
    out = _abi.lb_diag()
    st = L.lb_diagnostics_static(C.byref(desc), C.byref(params), C.c_void_p(dev.data_ptr()), int(step),
                                 C.c_void_p(solver.stream.cuda_stream), C.byref(out))
    _abi.check(st)
    return {"nu_side": list(out.nu_side), "nu_i": out.nu_i, "nu_o": out.nu_o, "nu_avg": out.nu_avg,
            "mass": out.mass, "mass_r": out.mass_r, "T_sum": out.T_sum, "u_max": out.u_max,
            "k_eq_i": out.k_eq_i, "k_eq_o": out.k_eq_o, "step": int(out.step), "status": int(out.status)}


def _cases():
    from paper_1806_10241_gb300 import workloads as W
    return [("cylinder_fp32", W.swirling_cylinder(nr=70, nz=96, Re=200.0, Ra=1e4, amp=1e-3, seed=2), "fp32"),
            ("annulus_fp64", W.annulus_convection(nr=33, nz=40, Ra=1e4, amp=1e-3, seed=4, swirl_inner=0.01),
             "fp64"),
            ("annulus_fp16", W.annulus_convection(nr=61, nz=45, Ra=1e4, amp=1e-3, seed=5), "fp16"),
            # the top split into a crystal and a free surface with the ramp: Nu over heated segments
            ("czochralski_fp32", W.czochralski(nr=60, nz=60, beta=0.4, Re_x=200.0, Re_c=-50.0, Pr=0.7, Gr=1e4),
             "fp32")]


@pytest.mark.parametrize("name,case,storage", _cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_static_scratch_diagnostics_match_lb_diagnostics(name, case, storage):
    from paper_1806_10241_gb300.solver import Solver
    s = Solver(case.params, storage=storage)
    s.init_fields(case.fields)
    for call in range(2):  # two calls in a row, on two different states
        s.step(150)
        want = s.diag()
        got = _static_diag(s, s.step_count)
        assert got["status"] == want["status"] == 0
        assert got["step"] == want["step"]
        for k in FIELDS:
            assert got[k] == pytest.approx(want[k], rel=1e-11, abs=1e-13), (name, call, k)
        for q in range(4):
            assert got["nu_side"][q] == pytest.approx(want["nu_side"][q], rel=1e-11, abs=1e-13)


def test_static_scratch_rejects_lattices_beyond_its_limit():
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300 import workloads as W
    L = _abi.load()
    case = W.swirling_cylinder(nr=4096, nz=30000)
    desc = _abi.make_desc(case.params, "fp32")
    params = _abi.make_params(case.params)
    out = _abi.lb_diag()
    fake = C.c_void_p(1 << 40)  # rejected before any device access
    st = L.lb_diagnostics_static(C.byref(desc), C.byref(params), fake, 0, None, C.byref(out))
    assert st == _abi.LB_ERR_ARG
    assert b"static array" in L.lb_last_error(None)
