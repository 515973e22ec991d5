"""ctypes binding of include/lb.h (argument marshalling only).

Every function keeps the C name.  The library is loaded from the in-tree
build (paper_1806_10241_gb300/_build/liblbaxi.so); if it is missing the import
fails loudly -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbaxi.so")

LB_OK, LB_ERR_ARG, LB_ERR_NOMEM, LB_ERR_CUDA, LB_ERR_DIVERGED, LB_ERR_TIMEOUT, LB_ERR_STATE = range(7)
LB_FP64, LB_FP32, LB_BF16, LB_FP16 = range(4)
STORAGE = {"fp64": LB_FP64, "fp32": LB_FP32, "bf16": LB_BF16, "fp16": LB_FP16}
STATUS_NAMES = {0: "LB_OK", 1: "LB_ERR_ARG", 2: "LB_ERR_NOMEM", 3: "LB_ERR_CUDA",
                4: "LB_ERR_DIVERGED", 5: "LB_ERR_TIMEOUT", 6: "LB_ERR_STATE"}


class lb_grid_desc(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nz", C.c_int32), ("r_inner", C.c_double),
                ("storage", C.c_int32), ("reserved", C.c_int32)]


class lb_side(C.Structure):
    _fields_ = [("flow", C.c_int32), ("swirl", C.c_int32), ("heat", C.c_int32),
                ("pad", C.c_int32), ("u_wx", C.c_double), ("u_wy", C.c_double),
                ("omega", C.c_double), ("T_w", C.c_double)]


class lb_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("omega3", C.c_double),
                ("omega_hi", C.c_double), ("g_beta", C.c_double), ("T0", C.c_double),
                ("body_fx", C.c_double), ("rho0", C.c_double), ("planar", C.c_int32),
                ("sign_literal", C.c_int32), ("explicit_sources", C.c_int32),
                ("pad", C.c_int32), ("side", lb_side * 4), ("top_split", C.c_int32), ("pad2", C.c_int32),
                ("top_outer", lb_side)]


class lb_diag(C.Structure):
    _fields_ = [("nu_side", C.c_double * 4), ("nu_i", C.c_double), ("nu_o", C.c_double),
                ("nu_avg", C.c_double), ("mass", C.c_double), ("mass_r", C.c_double),
                ("T_sum", C.c_double), ("u_max", C.c_double), ("step", C.c_int64),
                ("status", C.c_int32), ("pad", C.c_int32), ("k_eq_i", C.c_double),
                ("k_eq_o", C.c_double)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_st = C.c_int  # lb_status

# name -> (restype, argtypes): one entry per declaration in include/lb.h
PROTOTYPES = {
    "lb_required_bytes": (_st, [C.POINTER(lb_grid_desc), C.POINTER(C.c_size_t)]),
    "lb_create": (_st, [C.POINTER(lb_grid_desc), _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "lb_set_params": (_st, [_vp, C.POINTER(lb_params)]),
    "lb_init_fields": (_st, [_vp, _dp]),
    "lb_step": (_st, [_vp, C.c_int32]),
    "lb_get_fields": (_st, [_vp, _dp]),
    "lb_diagnostics": (_st, [_vp, C.POINTER(lb_diag)]),
    "lb_get_distributions": (_st, [_vp, _dp]),
    "lb_set_distributions": (_st, [_vp, _dp]),
    "lb_state_bytes": (_st, [_vp, C.POINTER(C.c_size_t)]),
    "lb_get_state": (_st, [_vp, _vp, C.c_size_t]),
    "lb_set_state": (_st, [_vp, _vp, C.c_size_t]),
    "lb_get_step": (_st, [_vp, C.POINTER(C.c_int64)]),
    "lb_set_launch": (_st, [_vp, C.c_int32, C.c_int32, C.c_int32]),
    "lb_get_launch": (_st, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lb_diagnostics_static": (_st, [C.POINTER(lb_grid_desc), C.POINTER(lb_params), _vp, C.c_int64, _vp,
                                    C.POINTER(lb_diag)]),
    "lb_batch_required_bytes": (_st, [C.c_int32, C.POINTER(C.c_size_t)]),
    "lb_batch_create": (_st, [C.POINTER(_vp), C.c_int32, _vp, C.c_size_t, _vp, C.POINTER(_vp)]),
    "lb_batch_set_launch": (_st, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "lb_selftest_timeout": (_st, [_vp, C.c_int32]),
    "lb_stream_function": (_st, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lb_batch_set_segments": (_st, [_vp, C.POINTER(C.c_int32)]),
    "lb_batch_get_occupancy": (_st, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "lb_batch_step": (_st, [_vp, C.c_int32]),
    "lb_batch_diagnostics": (_st, [_vp, _vp]),
    "lb_batch_destroy": (_st, [_vp]),
    "lb_destroy": (_st, [_vp]),
    "lb_last_error": (C.c_char_p, [_vp]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblbaxi.so (built by paper_1806_10241_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing: build it with paper_1806_10241_gb300.build.build()")
            L = C.CDLL(p)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx=None) -> None:
    if status != LB_OK:
        msg = load().lb_last_error(ctx).decode(errors="replace")
        raise LBError(status, msg)


def make_params(d: dict) -> lb_params:
    """lb_params from the parameter dict of a workload."""
    p = lb_params()
    p.nu = float(d["nu"])
    p.alpha = float(d["alpha"])
    p.omega3 = float(d.get("omega3", 1.0))
    p.omega_hi = float(d.get("omega_hi", 1.0))
    p.g_beta = float(d.get("g_beta", 0.0))
    p.T0 = float(d.get("T0", 0.0))
    p.body_fx = float(d.get("body_fx", 0.0))
    p.rho0 = float(d.get("rho0", 1.0))
    p.planar = int(d.get("planar", 0))
    p.sign_literal = int(d.get("sign_literal", 0))
    p.explicit_sources = int(d.get("explicit_sources", 0))
    def fill(dst, s):
        dst.flow = int(s.get("flow", 0))
        dst.swirl = int(s.get("swirl", 0))
        dst.heat = int(s.get("heat", 1))
        dst.u_wx = float(s.get("u_wx", 0.0))
        dst.u_wy = float(s.get("u_wy", 0.0))
        dst.omega = float(s.get("omega", 0.0))
        dst.T_w = float(s.get("T_w", 0.0))
    for i, s in enumerate(d["sides"]):
        fill(p.side[i], s)
    p.top_split = int(d.get("top_split", 0))
    if "top_outer" in d:
        fill(p.top_outer, d["top_outer"])
    return p


def make_desc(d: dict, storage: str | int) -> lb_grid_desc:
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return lb_grid_desc(int(d["nr"]), int(d["nz"]), float(d.get("r0", 0.0)), st, 0)
