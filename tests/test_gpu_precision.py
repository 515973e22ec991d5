"""16-bit storage against the FP64 oracle, on the heated swirling cylinder
(H/R = 2, lid u = 0.05, Ra = 1e5, Pr = 0.7).

The distributions are stored as FP16 (deviations scaled by 1024) or BF16
deviations from the rest state with stochastic rounding; the arithmetic is
FP32.  One rounding of a stored deviation has relative error at most u
(FP16 u = 2^-11, BF16 u = 2^-8); stochastic rounding keeps the per-step
errors from accumulating a bias, so the fields stay within a few u of the
oracle (bound used: 4 u in relative L2).  The FP32 path is held to the FP32
bar (relative L2 1e-5, Nu 1e-4).

Two cases:
  * the precision form of the benchmark cylinder on a 256 x 512 copy
    (Re = 1000 on R, nu = 0.0128), 1500 steps.  The Rayleigh-Benard layer is
    unstable here, and the storage rounding seeds the instability far above
    the 1e-6 initial perturbation, so Nu differs by more than the rounding
    itself: FP16 stays within 0.5 % of the oracle, BF16 within 2 %;
  * a viscous copy (128 x 256, Re = 125) where the flow follows the
    boundary forcing: Nu within 4 u of the oracle's, the bound the fields
    are held to.  The error of one run depends on its rounding sequence:
    builds whose arithmetic or random words differed gave 2e-6 to 7.6e-4
    (FP16) and 1e-4 to 9.6e-3 (BF16).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
CASES = {
    # name: (nr, nz, Re, steps, Nu tolerance per storage)
    "cylinder_256x512_Re1000": (256, 512, 1000.0, 1500, {"fp32": 1e-4, "fp16": 5e-3, "bf16": 2e-2}),
    "cylinder_128x256_Re125": (128, 256, 125.0, 2000, {"fp32": 1e-4, "fp16": 4 * U["fp16"], "bf16": 4 * U["bf16"]}),
}
_cache = {}


def _runs(name):
    if name in _cache:
        return _cache[name]
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_10241_gb300 import build
    build.build()
    import oracle
    from paper_1806_10241_gb300 import workloads as W
    from paper_1806_10241_gb300.solver import Solver
    nr, nz, Re, steps, _ = CASES[name]
    c = W.swirling_cylinder(nr=nr, nz=nz, Re=Re, Ra=1e5, Pr=0.7, u_lid=0.05, amp=1e-6, seed=0)
    o = oracle.Oracle(c.params)
    o.init_fields(c.fields)
    o.step(steps)
    out = {"oracle": (o.fields(), o.diag())}
    for storage in ("fp32", "fp16", "bf16"):
        s = Solver(c.params, storage=storage)
        s.init_fields(c.fields)
        s.step(steps)
        out[storage] = (s.fields(), s.diag())
    _cache.clear()
    _cache[name] = out
    return out


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_reduced_storage_fields_and_nusselt_against_oracle(name, storage):
    runs = _runs(name)
    fo, do = runs["oracle"]
    f, d = runs[storage]
    assert d["status"] == 0
    errs = {fld: _rel_l2(f[q], fo[q]) for q, fld in ((1, "u_z"), (2, "u_r"), (3, "u_theta"), (4, "T"))}
    nu_err = abs(d["nu_avg"] - do["nu_avg"]) / abs(do["nu_avg"])
    assert max(errs.values()) < (1e-5 if storage == "fp32" else 4 * U[storage]), (storage, errs)
    assert nu_err < CASES[name][4][storage], (storage, nu_err)
