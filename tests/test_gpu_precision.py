"""16-bit storage against the FP64 oracle: the precision form of the heated
swirling cylinder (H/R = 2, lid u = 0.05, Re = 1000, Ra = 1e5, Pr = 0.7) on
a 256 x 512 lattice.

The distributions are stored as FP16 (deviations scaled by 1024) or BF16
deviations from the rest state with stochastic rounding; the arithmetic is
FP32.  Tolerances follow from the storage precision: one rounding of a
stored deviation has relative error at most u (FP16 u = 2^-11, BF16
u = 2^-8); stochastic rounding keeps the per-step errors from accumulating a
bias, so the fields stay within a few u of the oracle (bound used: 4 u in
relative L2).  The average Nusselt number must stay within 0.5 % of the
oracle.  The FP32 path is held to the FP32 bar (relative L2 1e-5, Nu 1e-4).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STEPS = 1500
U = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()
    import oracle
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.solver import Solver
    c = W.swirling_cylinder(nr=256, nz=512, Re=1000.0, Ra=1e5, Pr=0.7, u_lid=0.05, amp=1e-6, seed=0)
    o = oracle.Oracle(c.params)
    o.init_fields(c.fields)
    o.step(STEPS)
    out = {"oracle": (o.fields(), o.diag())}
    for storage in ("fp32", "fp16", "bf16"):
        s = Solver(c.params, storage=storage)
        s.init_fields(c.fields)
        s.step(STEPS)
        out[storage] = (s.fields(), s.diag())
    return out


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_reduced_storage_fields_and_nusselt_against_oracle(runs, storage):
    fo, do = runs["oracle"]
    f, d = runs[storage]
    assert d["status"] == 0
    errs = {name: _rel_l2(f[q], fo[q]) for q, name in ((1, "u_z"), (2, "u_r"), (3, "u_theta"), (4, "T"))}
    nu_err = abs(d["nu_avg"] - do["nu_avg"]) / abs(do["nu_avg"])
    if storage == "fp32":
        assert max(errs.values()) < 1e-5, errs
        assert nu_err < 1e-4, nu_err
    else:
        assert max(errs.values()) < 4 * U[storage], (storage, errs)
        assert nu_err < 5e-3, (storage, nu_err)
