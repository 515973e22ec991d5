"""FP64 CPU oracle of the axisymmetric thermal cascaded LB method (arXiv 1806.10241).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_1806_10241_gb300``; the only
common ground is the numbers both are handed (parameters and initial fields).

The C source (``orc.c``) follows the paper equation by equation; this module
only compiles it with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

# side indices: 0 bottom (x=0), 1 top (x=H), 2 inner (y=r0), 3 outer (y=r0+nr)
FLOW_WALL, FLOW_AXIS, FLOW_PERIODIC, FLOW_FREE = 0, 1, 2, 3
SC_DIRICHLET, SC_NEUMANN, SC_AXIS, SC_PERIODIC, SC_RAMP = 0, 1, 2, 3, 4


class Side(C.Structure):
    _fields_ = [("flow", C.c_int32), ("swirl", C.c_int32), ("heat", C.c_int32),
                ("pad", C.c_int32), ("u_wx", C.c_double), ("u_wy", C.c_double),
                ("omega", C.c_double),
                ("T_w", C.c_double)]


class Params(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nz", C.c_int32), ("r0", C.c_double),
                ("nu", C.c_double), ("alpha", C.c_double), ("omega3", C.c_double),
                ("omega_hi", C.c_double), ("g_beta", C.c_double), ("T0", C.c_double),
                ("body_fx", C.c_double), ("rho0", C.c_double), ("planar", C.c_int32),
                ("sign_literal", C.c_int32), ("explicit_sources", C.c_int32),
                ("pad", C.c_int32), ("side", Side * 4), ("top_split", C.c_int32), ("pad2", C.c_int32),
                ("top_outer", Side)]


class Diag(C.Structure):
    _fields_ = [("nu_side", C.c_double * 4), ("nu_i", C.c_double), ("nu_o", C.c_double),
                ("nu_avg", C.c_double), ("mass", C.c_double), ("mass_r", C.c_double),
                ("T_sum", C.c_double), ("u_max", C.c_double), ("step", C.c_int64),
                ("k_eq_i", C.c_double), ("k_eq_o", C.c_double)]


def build(force: bool = False) -> str:
    """Compile orc.c into _build/liborc.so (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "orc.c")
    hdr = os.path.join(_HERE, "orc.h")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(Params)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            for name in ("orc_init_fields", "orc_set_dist"):
                getattr(L, name).argtypes = [C.c_void_p, dp]
            for name in ("orc_get_dist", "orc_fields"):
                getattr(L, name).argtypes = [C.c_void_p, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_diag_compute.argtypes = [C.c_void_p, C.POINTER(Diag)]
            L.orc_stream_function.argtypes = [C.c_void_p, dp, dp]
            L.orc_get_step.restype = C.c_int64
            L.orc_get_step.argtypes = [C.c_void_p]
            L.orc_eq_d2q9.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.orc_eq_d2q5.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.orc_collide_d2q9.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp, dp]
            L.orc_post_d2q9.argtypes = [dp, dp, dp]
            L.orc_collide_d2q5.argtypes = [dp, C.c_double, C.c_double, C.c_double, dp, C.c_int, dp]
            L.orc_post_d2q5.argtypes = [dp, dp, dp]
            _lib = L
        return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(d: dict) -> Params:
    """Build the C parameter struct from a plain dict (see workloads)."""
    p = Params()
    for k in ("nr", "nz"):
        setattr(p, k, int(d[k]))
    for k, dflt in (("r0", 0.0), ("nu", None), ("alpha", None), ("omega3", 1.0),
                    ("omega_hi", 1.0), ("g_beta", 0.0), ("T0", 0.0), ("body_fx", 0.0),
                    ("rho0", 1.0)):
        v = d.get(k, dflt)
        if v is None:
            raise KeyError(k)
        setattr(p, k, float(v))
    p.planar = int(d.get("planar", 0))
    p.sign_literal = int(d.get("sign_literal", 0))
    p.explicit_sources = int(d.get("explicit_sources", 0))
    def fill(dst, s):
        dst.flow = int(s.get("flow", FLOW_WALL))
        dst.swirl = int(s.get("swirl", SC_DIRICHLET))
        dst.heat = int(s.get("heat", SC_NEUMANN))
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


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


class Oracle:
    """One lattice advanced by the FP64 oracle."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        self.nr, self.nz = self._p.nr, self._p.nz
        h = lib().orc_create(C.byref(self._p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return self.nr * self.nz

    def init_fields(self, fields: np.ndarray) -> None:
        a = np.ascontiguousarray(fields, dtype=np.float64).reshape(5, self.nz, self.nr)
        lib().orc_init_fields(self._h, _dp(a))

    def set_dist(self, d: np.ndarray) -> None:
        a = np.ascontiguousarray(d, dtype=np.float64).reshape(19, self.nz, self.nr)
        lib().orc_set_dist(self._h, _dp(a))

    def get_dist(self) -> np.ndarray:
        a = np.empty((19, self.nz, self.nr), np.float64)
        lib().orc_get_dist(self._h, _dp(a))
        return a

    def step(self, n: int = 1) -> None:
        lib().orc_step(self._h, int(n))

    def fields(self) -> np.ndarray:
        """[5, nz, nr]: rho, u_x (axial), u_y (radial), u_theta, T of the
        pre-collision state the next step would collide."""
        a = np.empty((5, self.nz, self.nr), np.float64)
        lib().orc_fields(self._h, _dp(a))
        return a

    def diag(self) -> dict:
        d = Diag()
        lib().orc_diag_compute(self._h, C.byref(d))
        return {"nu_side": list(d.nu_side), "nu_i": d.nu_i, "nu_o": d.nu_o,
                "nu_avg": d.nu_avg, "mass": d.mass, "mass_r": d.mass_r,
                "T_sum": d.T_sum, "u_max": d.u_max, "k_eq_i": d.k_eq_i, "k_eq_o": d.k_eq_o,
                "step": int(d.step)}

    def stream_function(self) -> tuple:
        """(psi [nz, nr] on the cell faces y = r0 + j + 1, max |psi|)."""
        a = np.empty((self.nz, self.nr), np.float64)
        m = C.c_double()
        lib().orc_stream_function(self._h, _dp(a), C.byref(m))
        return a, m.value

    @property
    def step_count(self) -> int:
        return int(lib().orc_get_step(self._h))


# ---- per-node building blocks (for the brute-force pins) -------------------

def eq_d2q9(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_eq_d2q9(rho, ux, uy, _dp(out))
    return out


def eq_d2q5(s, ux, uy) -> np.ndarray:
    out = np.zeros(5)
    lib().orc_eq_d2q5(s, ux, uy, _dp(out))
    return out


def collide_d2q9(f, rho, ux, uy, om) -> np.ndarray:
    f = np.ascontiguousarray(f, np.float64)
    om = np.ascontiguousarray(om, np.float64)
    out = np.zeros(9)
    lib().orc_collide_d2q9(_dp(f), rho, ux, uy, _dp(om), _dp(out))
    return out


def post_d2q9(f, ph) -> np.ndarray:
    f = np.ascontiguousarray(f, np.float64)
    ph = np.ascontiguousarray(ph, np.float64)
    out = np.zeros(9)
    lib().orc_post_d2q9(_dp(f), _dp(ph), _dp(out))
    return out


def collide_d2q5(g, s, ux, uy, om, sign_literal=0) -> np.ndarray:
    g = np.ascontiguousarray(g, np.float64)
    om = np.ascontiguousarray(om, np.float64)
    out = np.zeros(5)
    lib().orc_collide_d2q5(_dp(g), s, ux, uy, _dp(om), int(sign_literal), _dp(out))
    return out


def post_d2q5(g, qh) -> np.ndarray:
    g = np.ascontiguousarray(g, np.float64)
    qh = np.ascontiguousarray(qh, np.float64)
    out = np.zeros(5)
    lib().orc_post_d2q5(_dp(g), _dp(qh), _dp(out))
    return out
