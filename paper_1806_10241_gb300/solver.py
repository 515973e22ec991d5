"""One lattice on the GPU through the C ABI.

PyTorch supplies the device buffer and the CUDA stream; every step of the
method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def required_bytes(params: dict, storage: str = "fp32") -> int:
    L = _abi.load()
    n = C.c_size_t()
    desc = _abi.make_desc(params, storage)
    _abi.check(L.lb_required_bytes(C.byref(desc), C.byref(n)))
    return int(n.value)


def diag_dict(d) -> dict:
    """lb_diag as a dict."""
    return {"nu_side": list(d.nu_side), "nu_i": d.nu_i, "nu_o": d.nu_o, "nu_avg": d.nu_avg,
            "mass": d.mass, "mass_r": d.mass_r, "T_sum": d.T_sum, "u_max": d.u_max,
            "k_eq_i": d.k_eq_i, "k_eq_o": d.k_eq_o, "step": int(d.step), "status": int(d.status)}


class Solver:
    """A lattice whose distributions live on `device`.

    params: the workload parameter dict (see workloads).  storage: "fp64",
    "fp32", "bf16" or "fp16".  stream: a torch.cuda.Stream (default: the
    current stream).  buffer: optional preallocated uint8 CUDA tensor.
    """

    def __init__(self, params: dict, storage: str = "fp32", device: str | torch.device = "cuda",
                 stream: torch.cuda.Stream | None = None, buffer: torch.Tensor | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device")
        self.L = _abi.load()
        self.params = dict(params)
        self.storage = storage
        self.nr, self.nz = int(params["nr"]), int(params["nz"])
        self.device = torch.device(device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.nbytes = required_bytes(params, storage)
        if buffer is None:
            buffer = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        if buffer.numel() < self.nbytes:
            raise ValueError("buffer too small")
        self.buffer = buffer
        desc = _abi.make_desc(params, storage)
        ctx = C.c_void_p()
        _abi.check(self.L.lb_create(C.byref(desc), C.c_void_p(buffer.data_ptr()),
                                    buffer.numel(), C.c_void_p(self.stream.cuda_stream),
                                    C.byref(ctx)))
        self.ctx = ctx
        self._p = _abi.make_params(params)
        self._check(self.L.lb_set_params(self.ctx, C.byref(self._p)))

    # -- plumbing -------------------------------------------------------------
    def _check(self, st: int) -> None:
        _abi.check(st, self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.L.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return self.nr * self.nz

    # -- the ABI --------------------------------------------------------------
    def set_launch(self, seg_rows: int = 0, warps_per_block: int = 0, row_fetch: int = 0) -> None:
        """row_fetch: 0 automatic, 1 plain loads, 2 TMA ring, 3 TMA ring with
        the rows read in place (FP32 / 16-bit storage)."""
        self._check(self.L.lb_set_launch(self.ctx, int(seg_rows), int(warps_per_block), int(row_fetch)))

    def get_launch(self) -> tuple:
        """(seg_rows, warps_per_block, row_fetch) the next step uses."""
        s, w, f = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.L.lb_get_launch(self.ctx, C.byref(s), C.byref(w), C.byref(f)))
        return s.value, w.value, f.value

    def reset(self) -> None:
        """lb_set_params again: the state returns to rest at step 0 and the
        device status word is cleared."""
        self._check(self.L.lb_set_params(self.ctx, C.byref(self._p)))

    def init_fields(self, fields: np.ndarray) -> None:
        a = np.ascontiguousarray(fields, np.float64).reshape(5, self.nz, self.nr)
        self._check(self.L.lb_init_fields(self.ctx, _dptr(a)))

    def step(self, n: int = 1) -> None:
        self._check(self.L.lb_step(self.ctx, int(n)))

    def fields(self, out: np.ndarray | None = None) -> np.ndarray:
        """[5, nz, nr] rho, u_x, u_y, u_theta, T; `out` may be a (pinned)
        float64 array of that shape to receive them."""
        a = np.empty((5, self.nz, self.nr), np.float64) if out is None else out
        if a.shape != (5, self.nz, self.nr) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array of shape (5, nz, nr)")
        self._check(self.L.lb_get_fields(self.ctx, _dptr(a)))
        return a

    def diag(self) -> dict:
        d = _abi.lb_diag()
        self._check(self.L.lb_diagnostics(self.ctx, C.byref(d)))
        return diag_dict(d)

    def stream_function(self, field: bool = False) -> tuple:
        """(psi [nz, nr] on the cell faces y = r0 + j + 1 or None, max |psi|)."""
        a = np.empty((self.nz, self.nr), np.float64) if field else None
        m = C.c_double()
        self._check(self.L.lb_stream_function(self.ctx, _dptr(a) if field else None, C.byref(m)))
        return a, m.value

    def get_dist(self) -> np.ndarray:
        a = np.empty((19, self.nz, self.nr), np.float64)
        self._check(self.L.lb_get_distributions(self.ctx, _dptr(a)))
        return a

    def set_dist(self, d: np.ndarray) -> None:
        a = np.ascontiguousarray(d, np.float64).reshape(19, self.nz, self.nr)
        self._check(self.L.lb_set_distributions(self.ctx, _dptr(a)))

    def state_bytes(self) -> int:
        n = C.c_size_t()
        self._check(self.L.lb_state_bytes(self.ctx, C.byref(n)))
        return int(n.value)

    def get_state(self) -> bytes:
        n = self.state_bytes()
        buf = C.create_string_buffer(n)
        self._check(self.L.lb_get_state(self.ctx, buf, n))
        return buf.raw

    def set_state(self, blob: bytes) -> None:
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.L.lb_set_state(self.ctx, buf, len(blob)))

    @property
    def step_count(self) -> int:
        s = C.c_int64()
        self._check(self.L.lb_get_step(self.ctx, C.byref(s)))
        return int(s.value)
