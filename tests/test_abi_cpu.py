"""The C ABI library loads and exports what include/lb.h declares (CPU only).

No compute call is made: only the host-side argument checks run.
"""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1806_10241_gb300 import _abi, build
    build.build()
    return _abi.load()


def declared():
    txt = open(HEADER).read()
    return re.findall(r"LB_EXPORT\s+(?:lb_status|const char \*)\s*(lb_\w+)\s*\(", txt)


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1806_10241_gb300 import _abi
    names = declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.PROTOTYPES, n
    assert set(_abi.PROTOTYPES) == set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lb_\w+)", out))
    assert exported == set(names)


def test_struct_layouts_match_the_header(tmp_path):
    from paper_1806_10241_gb300 import _abi
    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lb.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(lb_grid_desc), sizeof(lb_side), sizeof(lb_params), sizeof(lb_diag));
  printf("%zu %zu %zu %zu\\n", offsetof(lb_params, side), offsetof(lb_diag, step), offsetof(lb_diag, status),
         offsetof(lb_diag, k_eq_i));
  return 0; }
""")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    sizes = list(map(int, a.split()))
    offs = list(map(int, b.split()))
    assert sizes == [C.sizeof(_abi.lb_grid_desc), C.sizeof(_abi.lb_side), C.sizeof(_abi.lb_params),
                     C.sizeof(_abi.lb_diag)]
    assert offs == [_abi.lb_params.side.offset, _abi.lb_diag.step.offset, _abi.lb_diag.status.offset,
                    _abi.lb_diag.k_eq_i.offset]


def test_required_bytes_and_argument_checks(lib):
    from paper_1806_10241_gb300 import _abi
    n = C.c_size_t()
    d = _abi.lb_grid_desc(1024, 2048, 0.0, _abi.LB_FP32, 0)
    assert lib.lb_required_bytes(C.byref(d), C.byref(n)) == _abi.LB_OK
    dist = 19 * 2048 * 1024 * 4
    assert 2 * dist <= n.value <= 2 * dist + (1 << 20)
    d16 = _abi.lb_grid_desc(1024, 2048, 0.0, _abi.LB_FP16, 0)
    n16 = C.c_size_t()
    assert lib.lb_required_bytes(C.byref(d16), C.byref(n16)) == _abi.LB_OK
    assert n16.value < 0.51 * n.value + (1 << 20)
    for bad in (_abi.lb_grid_desc(1, 8, 0.0, 1, 0), _abi.lb_grid_desc(8, 1, 0.0, 1, 0),
                _abi.lb_grid_desc(8, 8, -1.0, 1, 0), _abi.lb_grid_desc(8, 8, 0.0, 7, 0),
                _abi.lb_grid_desc(8, 8, 0.0, 1, 3)):
        assert lib.lb_required_bytes(C.byref(bad), C.byref(n)) == _abi.LB_ERR_ARG
        assert len(lib.lb_last_error(None)) > 0


def test_create_and_parameter_validation_without_device_work(lib):
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300 import workloads as W
    case = W.swirling_cylinder(nr=16, nz=32)
    d = _abi.make_desc(case.params, "fp32")
    n = C.c_size_t()
    lib.lb_required_bytes(C.byref(d), C.byref(n))
    ctx = C.c_void_p()
    fake = C.c_void_p(1 << 40)  # aligned, never dereferenced on this path
    assert lib.lb_create(C.byref(d), fake, n.value - 256, None, C.byref(ctx)) == _abi.LB_ERR_NOMEM
    assert lib.lb_create(C.byref(d), C.c_void_p((1 << 40) + 8), n.value, None, C.byref(ctx)) == _abi.LB_ERR_ARG
    assert lib.lb_create(C.byref(d), fake, n.value, None, C.byref(ctx)) == _abi.LB_OK
    try:
        assert lib.lb_step(ctx, 1) == _abi.LB_ERR_STATE
        bad = dict(case.params)
        bad["nu"] = -1.0
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(bad))) == _abi.LB_ERR_ARG
        bad = dict(case.params)
        bad["sides"] = [dict(s) for s in case.params["sides"]]
        bad["sides"][3]["flow"] = W.FLOW_AXIS  # axis on the outer side
        bad["sides"][3]["swirl"] = bad["sides"][3]["heat"] = W.SC_AXIS
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(bad))) == _abi.LB_ERR_ARG
        bad = dict(case.params)
        bad["sides"] = [dict(s) for s in case.params["sides"]]
        bad["sides"][0]["flow"] = W.FLOW_PERIODIC  # only one end periodic
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(bad))) == _abi.LB_ERR_ARG
        assert b"periodic" in lib.lb_last_error(ctx)
        # the Czochralski family (Sec. 3.6): a free surface only on an end wall, the
        # ramp only on the top's outer segment, the split inside the lattice
        bad = dict(case.params)
        bad["sides"] = [dict(s) for s in case.params["sides"]]
        bad["sides"][3]["flow"] = W.FLOW_FREE
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(bad))) == _abi.LB_ERR_ARG
        assert b"free surface" in lib.lb_last_error(ctx)
        bad = dict(case.params)
        bad["sides"] = [dict(s) for s in case.params["sides"]]
        bad["sides"][1]["heat"] = W.SC_RAMP
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(bad))) == _abi.LB_ERR_ARG
        assert b"ramp" in lib.lb_last_error(ctx)
        cz = W.czochralski(nr=16, nz=32)
        for key, val in (("top_split", 16), ("top_split", -1)):
            assert lib.lb_set_params(ctx, C.byref(_abi.make_params(dict(cz.params, **{key: val})))) == _abi.LB_ERR_ARG
        outer = dict(cz.params["top_outer"], flow=W.FLOW_AXIS)
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(dict(cz.params, top_outer=outer)))) == _abi.LB_ERR_ARG
        outer = dict(cz.params["top_outer"], T_w=float("nan"))
        assert lib.lb_set_params(ctx, C.byref(_abi.make_params(dict(cz.params, top_outer=outer)))) == _abi.LB_ERR_ARG
        assert lib.lb_set_launch(ctx, 16, 9, 0) == _abi.LB_ERR_ARG
        assert lib.lb_set_launch(ctx, 16, 4, 4) == _abi.LB_ERR_ARG
        seg, wpb, fetch = C.c_int32(), C.c_int32(), C.c_int32()
        assert lib.lb_set_launch(ctx, 5, 2, 2) == _abi.LB_OK
        assert lib.lb_get_launch(ctx, C.byref(seg), C.byref(wpb), C.byref(fetch)) == _abi.LB_OK
        assert (seg.value, wpb.value, fetch.value) == (5, 2, 2)
        assert lib.lb_set_launch(ctx, 0, 0, 0) == _abi.LB_OK  # automatic: the resident-row TMA ring
        assert lib.lb_get_launch(ctx, C.byref(seg), C.byref(wpb), C.byref(fetch)) == _abi.LB_OK
        assert seg.value > 0 and 1 <= wpb.value <= 8 and fetch.value == 3
        assert lib.lb_get_launch(None, None, None, None) == _abi.LB_ERR_ARG
        s = C.c_int64()
        assert lib.lb_get_step(ctx, C.byref(s)) == _abi.LB_OK and s.value == 0
    finally:
        assert lib.lb_destroy(ctx) == _abi.LB_OK


def test_default_launch_respects_the_grid_limit_for_tall_lattices(lib):
    """The default 6-row segments of 16-bit storage would need more than 65535
    z-blocks for nz = 400000."""
    from paper_1806_10241_gb300 import _abi
    from paper_1806_10241_gb300 import workloads as W
    params = dict(W.swirling_cylinder(nr=64, nz=8).params, nz=400000)  # parameters only, no fields
    d = _abi.make_desc(params, "fp16")
    n = C.c_size_t()
    assert lib.lb_required_bytes(C.byref(d), C.byref(n)) == _abi.LB_OK
    ctx = C.c_void_p()
    assert lib.lb_create(C.byref(d), C.c_void_p(1 << 40), n.value, None, C.byref(ctx)) == _abi.LB_OK
    try:
        seg, wpb, fetch = C.c_int32(), C.c_int32(), C.c_int32()
        assert lib.lb_get_launch(ctx, C.byref(seg), C.byref(wpb), C.byref(fetch)) == _abi.LB_OK
        assert (400000 + seg.value - 1) // seg.value <= 65535
    finally:
        lib.lb_destroy(ctx)
